// k_traj.cu -- the trajectory-optimisation ends of the whole-body evaluation:
// joint states from uniform cubic B-spline control points (Sec. 4,
// Eq. bspline-cubic) with the boundary conditions of Sec. 4.2, the
// control-point gradient (Eq. backward_grad), and the
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
#include "spline_basis.cuh"

namespace wbe {

// Boundary conditions (Sec. 4.2).  The spline is evaluated on an extended
// knot sequence of Kx = K + 3 hs + 3 es knots: with a start state (hs = 1)
// the ghost knots u_-3, u_-2, u_-1 of Eqs. fixed_3, fixed_2, fixed_1 come
// first,
//   u_-3 = th0 - a0 dt^2 / 6,  u_-2 = th0 + v0 dt + a0 dt^2 / 3,
//   u_-1 = th0 + 2 v0 dt + 11 a0 dt^2 / 6,
// and for a static goal (es = 1) the last control point is repeated three
// more times.  Samples spread over the Kx - 3 segments of the extended
// sequence; with hs = es = 0 it is U itself.
struct Knots {
  const float* u;   // the K control points of one (trajectory, joint)
  const float* st;  // theta_0, thetadot_0, thetaddot_0 of it, or nullptr
  int K, hs;
  float dt;
  __device__ __forceinline__ float operator()(int x) const {
    const int r = x - 3 * hs;
    if (r >= K) return __ldg(u + K - 1);
    if (r >= 0) return __ldg(u + r);
    const float th = __ldg(st), v = __ldg(st + 1), a = __ldg(st + 2);
    const float a2 = a * dt * dt;
    if (r == -3) return fmaf(-1.0f / 6.0f, a2, th);
    if (r == -2) return fmaf(1.0f / 3.0f, a2, fmaf(v, dt, th));
    return fmaf(11.0f / 6.0f, a2, fmaf(2.0f * v, dt, th));
  }
};

// one thread per (joint, configuration); b fastest so that stores coalesce
__global__ void __launch_bounds__(256) bspline_fwd_kernel(int64_t n_traj, int d, int K, int T,
                                                          float dt, const float* __restrict__ U,
                                                          const float* __restrict__ start,
                                                          int es, float* q, float* qd,
                                                          float* qdd) {
  const int64_t B = n_traj * T;
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= B * d) return;
  const int j = (int)(idx / B);
  const int64_t b = idx - (int64_t)j * B;
  const int64_t tr = b / T;
  const int s = (int)(b - tr * T);
  const int hs = start != nullptr;
  const int Kx = K + 3 * hs + 3 * es;
  int k;
  float a;
  bs_sample(s, Kx, T, k, a);
  float Bm[3][4];
  bs_basis(a, dt, Bm);
  const Knots kn{U + (tr * d + j) * K, hs ? start + (tr * d + j) * 3 : nullptr, K, hs, dt};
  const float u0 = kn(k), u1 = kn(k + 1), u2 = kn(k + 2), u3 = kn(k + 3);
  float out[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    out[r] = fmaf(Bm[r][3], u3, fmaf(Bm[r][2], u2, fmaf(Bm[r][1], u1, Bm[r][0] * u0)));
  const int64_t o = (int64_t)j * B + b;
  if (q) q[o] = out[0];
  if (qd) qd[o] = out[1];
  if (qdd) qdd[o] = out[2];
}

// Gradient of extended knot x of one (trajectory, joint): the sum of
// B(alpha_s)^T g_s over the samples of segments x-3 .. x in sample order.
struct KnotGrad {
  const float* tab;  // [T][12] basis rows
  const int* first;  // [nseg + 1] first sample of each segment
  int nseg;
  const float *gq, *gqd, *gqdd, *gqd2, *gqdd2;  // already offset to (joint, trajectory)
  __device__ __forceinline__ float operator()(int x) const {
    const int m0 = max(x - 3, 0), m1 = min(x, nseg - 1);
    float acc = 0.0f;
    if (m0 <= m1) {
      int m = m0;
      for (int s = first[m0]; s < first[m1 + 1]; ++s) {
        while (s >= first[m + 1]) ++m;  // segment of sample s
        const int l = x - m;            // this knot's place in the window
        const float* Bs = tab + s * 12;
        float c = 0.0f;
        if (gq) c = fmaf(Bs[l], __ldg(gq + s), c);
        float gv = gqd ? __ldg(gqd + s) : 0.0f;  // the two qd gradients add
        if (gqd2) gv += __ldg(gqd2 + s);
        c = fmaf(Bs[4 + l], gv, c);
        float ga = gqdd ? __ldg(gqdd + s) : 0.0f;
        if (gqdd2) ga += __ldg(gqdd2 + s);
        c = fmaf(Bs[8 + l], ga, c);
        acc += c;
      }
    }
    return acc;
  }
};

// One thread per control point (trajectory, joint, k), plus with a start
// state one per (trajectory, joint) for the start-state gradient (no atomics,
// deterministic).  The basis rows and segment of every sample and the first
// sample of every segment are tabled in shared memory per block.  With a
// static goal the last control point also sums the gradients of its three
// repeats; the start-state gradient is the transpose of the ghost knots'
// linear map applied to their three gradients.
__global__ void __launch_bounds__(256) bspline_bwd_kernel(
    int64_t n_traj, int d, int K, int T, float dt, int hs, int es, const float* __restrict__ gq,
    const float* __restrict__ gqd, const float* __restrict__ gqdd,
    const float* __restrict__ gqd2, const float* __restrict__ gqdd2, float* gU,
    float* gstart) {
  extern __shared__ float tab[];  // [T][12] basis rows, then [Kx-2] first samples
  int* first = reinterpret_cast<int*>(tab + (size_t)T * 12);
  const int Kx = K + 3 * hs + 3 * es;
  const int nseg = Kx - 3;
  for (int s = threadIdx.x; s < T; s += blockDim.x) {
    int k;
    float a;
    bs_sample(s, Kx, T, k, a);
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
  const int per = K + hs;  // threads per (trajectory, joint)
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n_traj * d * per) return;
  const int64_t tj = idx / per;  // trajectory * d + joint
  const int t = (int)(idx - tj * per);
  const int64_t tr = tj / d;
  const int j = (int)(tj - tr * d);
  const int64_t base = (int64_t)j * B + tr * T;
  const KnotGrad kg{tab, first, nseg, gq ? gq + base : nullptr, gqd ? gqd + base : nullptr,
                    gqdd ? gqdd + base : nullptr, gqd2 ? gqd2 + base : nullptr,
                    gqdd2 ? gqdd2 + base : nullptr};
  if (t < hs) {  // the start-state gradient through u_-3, u_-2, u_-1
    const float g3 = kg(0), g2 = kg(1), g1 = kg(2);
    if (gstart) {
      float* o = gstart + tj * 3;
      o[0] = g3 + g2 + g1;
      o[1] = dt * fmaf(2.0f, g1, g2);
      o[2] = dt * dt * fmaf(11.0f / 6.0f, g1, fmaf(1.0f / 3.0f, g2, (-1.0f / 6.0f) * g3));
    }
    return;
  }
  const int k = t - hs;
  const int x = k + 3 * hs;
  float acc = kg(x);
  if (es && k == K - 1)
    for (int r = 1; r <= 3; ++r) acc += kg(x + r);
  gU[tj * K + k] = acc;
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
                               const float* start, int end_static, float* q, float* qd,
                               float* qdd, cudaStream_t s) {
  const int64_t n = n_traj * T * d;
  bspline_fwd_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n_traj, d, K, T, dt, U, start,
                                                                 end_static ? 1 : 0, q, qd, qdd);
  return cudaGetLastError();
}

size_t bspline_bwd_smem(int Kx, int T) {
  return sizeof(float) * (size_t)T * 12 + sizeof(int) * (size_t)(Kx - 2);
}

cudaError_t launch_bspline_bwd(int64_t n_traj, int d, int K, int T, float dt, int has_start,
                               int end_static, const float* gq, const float* gqd,
                               const float* gqdd, const float* gqd2, const float* gqdd2,
                               float* gU, float* gstart, cudaStream_t s) {
  const int hs = has_start ? 1 : 0, es = end_static ? 1 : 0;
  const size_t smem = bspline_bwd_smem(K + 3 * hs + 3 * es, T);
  cudaError_t e = cudaFuncSetAttribute(bspline_bwd_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t n = n_traj * d * (K + hs);
  bspline_bwd_kernel<<<(unsigned)((n + 255) / 256), 256, smem, s>>>(
      n_traj, d, K, T, dt, hs, es, gq, gqd, gqdd, gqd2, gqdd2, gU, gstart);
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
