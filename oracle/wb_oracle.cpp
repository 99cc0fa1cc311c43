// wb_oracle.cpp -- plain FP64 CPU oracle for the whole-body evaluation.
//
// TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
// benchmark's CPU-baseline leg may load this library.  It shares no code,
// header, table or helper with the CUDA library and does not include it.
//
// What it computes, per configuration (the evaluation of Sec. 6 of the paper):
//   1. forward kinematics over the kinematic tree (Sec. 6.1.1): for k in index
//      order, T_k = T_parent(k) * T_fixed,k * J_k(theta_k), with
//      theta_k = mimic_mult_k * q[jidx_k] + mimic_off_k (mimic joints, Fig. 3b);
//   2. collision-sphere centres c_s = R_link(s) c_local,s + p_link(s) (Sec. 6.1.1);
//   3. self-collision (Sec. 6.2) by brute force over every masked pair:
//      d_ij = |c_i - c_j| - r_i - r_j, d_min = min d_ij, worst = the smallest
//      pair index attaining it, colliding_ij = (d_ij < 0);
//   4. inverse dynamics by the recursive Newton-Euler algorithm (Sec. 6.3,
//      Alg. 4) written with full 6x6 Plucker matrices (Featherstone's spatial
//      algebra): velocity/acceleration sweep base->tips, per-link force,
//      force sweep tips->base, tau_j += m_k S_k^T f_k.
//   5. gradients of L = <g_pose,poses> + <g_sph,centres> + g_dmin*d_min +
//      <g_tau,tau> with respect to q, qd, qdd by forward-mode dual numbers
//      (one pass per input coordinate); d_min differentiates through the
//      selected worst pair.
//   6. the uniform cubic B-spline of Sec. 4 (Eq. bspline-cubic), used to make
//      joint trajectories from control points, and its vector-Jacobian
//      product with respect to the control points (Eq. backward_grad);
//   7. kinematic Jacobians of chosen links and the whole-body centre of mass
//      with its Jacobian, by dual-number differentiation of step 1.
//
// Readings where the paper is silent: gravity enters as a fictitious base
// acceleration a_base = [0; -g]; a fixed joint has an empty motion subspace;
// spatial inertia at the link origin comes from (mass, CoM, inertia about the
// CoM) by the parallel-axis theorem; payload point masses add their own 6x6
// spatial inertia to their link.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

// ---------------------------------------------------------------------------
// forward-mode dual number
// ---------------------------------------------------------------------------
struct Dual {
  double v, d;
  Dual(double x = 0.0, double dx = 0.0) : v(x), d(dx) {}
};
static inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
static inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
static inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
static inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
static inline Dual operator/(Dual a, Dual b) {
  return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
static inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
static inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
static inline Dual sin(Dual a) { return Dual(std::sin(a.v), std::cos(a.v) * a.d); }
static inline Dual cos(Dual a) { return Dual(std::cos(a.v), -std::sin(a.v) * a.d); }
static inline Dual sqrt(Dual a) {
  double s = std::sqrt(a.v);
  return Dual(s, s > 0 ? a.d / (2.0 * s) : 0.0);
}
static inline double val(double x) { return x; }
static inline double val(const Dual& x) { return x.v; }

// ---------------------------------------------------------------------------
// robot descriptor (C ABI, arrays owned by the caller)
// ---------------------------------------------------------------------------
extern "C" {
struct or_robot {
  int n, d, S, P, n_pm;
  const int* parent;        // [n], -1 = world, parent[k] < k
  const int* jtype;         // [n], 0 fixed, 1 revolute, 2 prismatic
  const double* axis;       // [n][3], joint axis in the link frame
  const double* T_fixed;    // [n][12], R row-major then p
  const int* jidx;          // [n], -1 for fixed
  const double* mimic_mult; // [n]
  const double* mimic_off;  // [n]
  const double* gravity;    // [3]
  const int* sph_link;      // [S]
  const double* sph_c;      // [S][3]
  const double* sph_r;      // [S]
  const int* pairs;         // [P][2]
  const double* mass;       // [n]
  const double* com;        // [n][3]
  const double* Icom;       // [n][6] xx yy zz xy xz yz
  const int* pm_link;       // [n_pm]
  const double* pm_mass;    // [n_pm]
  const double* pm_pos;     // [n_pm][3]
};
}

// ---------------------------------------------------------------------------
// 3x3 and 6x6 helpers (plain loops)
// ---------------------------------------------------------------------------
template <class T> struct M3 { T a[3][3]; };
template <class T> struct M6 { T a[6][6]; };

template <class T> static M3<T> m3_mul(const M3<T>& A, const M3<T>& B) {
  M3<T> C;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s = 0.0;
      for (int k = 0; k < 3; ++k) s += A.a[i][k] * B.a[k][j];
      C.a[i][j] = s;
    }
  return C;
}
template <class T> static void m3_vec(const M3<T>& A, const T* x, T* y) {
  for (int i = 0; i < 3; ++i) y[i] = A.a[i][0] * x[0] + A.a[i][1] * x[1] + A.a[i][2] * x[2];
}
template <class T> static M3<T> m3_eye() {
  M3<T> I;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) I.a[i][j] = (i == j) ? 1.0 : 0.0;
  return I;
}
template <class T> static M3<T> m3_T(const M3<T>& A) {
  M3<T> B;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) B.a[i][j] = A.a[j][i];
  return B;
}
// skew matrix [x]^ with [x]^ y = x cross y
template <class T> static M3<T> skew(const T* x) {
  M3<T> S;
  S.a[0][0] = 0.0;  S.a[0][1] = -x[2]; S.a[0][2] = x[1];
  S.a[1][0] = x[2]; S.a[1][1] = 0.0;   S.a[1][2] = -x[0];
  S.a[2][0] = -x[1]; S.a[2][1] = x[0]; S.a[2][2] = 0.0;
  return S;
}
// rotation by angle t about unit axis k (Rodrigues' formula)
template <class T> static M3<T> rodrigues(const double* k, T t) {
  T kk[3] = {T(k[0]), T(k[1]), T(k[2])};
  M3<T> K = skew(kk), K2 = m3_mul(K, K), R = m3_eye<T>();
  T s = sin(t), c = cos(t);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R.a[i][j] = R.a[i][j] + s * K.a[i][j] + (T(1.0) - c) * K2.a[i][j];
  return R;
}

template <class T> static M6<T> m6_zero() {
  M6<T> A;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) A.a[i][j] = 0.0;
  return A;
}
template <class T> static M6<T> m6_mul(const M6<T>& A, const M6<T>& B) {
  M6<T> C;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) {
      T s = 0.0;
      for (int k = 0; k < 6; ++k) s += A.a[i][k] * B.a[k][j];
      C.a[i][j] = s;
    }
  return C;
}
template <class T> static void m6_vec(const M6<T>& A, const T* x, T* y) {
  for (int i = 0; i < 6; ++i) {
    T s = 0.0;
    for (int k = 0; k < 6; ++k) s += A.a[i][k] * x[k];
    y[i] = s;
  }
}
template <class T> static void m6T_vec(const M6<T>& A, const T* x, T* y) {
  for (int i = 0; i < 6; ++i) {
    T s = 0.0;
    for (int k = 0; k < 6; ++k) s += A.a[k][i] * x[k];
    y[i] = s;
  }
}
// Plucker transform from parent to child coordinates for a child frame with
// rotation E (parent->child coordinates) whose origin sits at r (parent coords):
// X = [E 0; -E [r]^ E]
template <class T> static M6<T> plucker(const M3<T>& E, const T* r) {
  M6<T> X = m6_zero<T>();
  M3<T> Er = m3_mul(E, skew(r));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      X.a[i][j] = E.a[i][j];
      X.a[i + 3][j + 3] = E.a[i][j];
      X.a[i + 3][j] = -Er.a[i][j];
    }
  return X;
}
// motion cross-product matrix crm(v) = [[w]^ 0; [u]^ [w]^]
template <class T> static M6<T> crm(const T* v) {
  M6<T> C = m6_zero<T>();
  M3<T> W = skew(v), U = skew(v + 3);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      C.a[i][j] = W.a[i][j];
      C.a[i + 3][j + 3] = W.a[i][j];
      C.a[i + 3][j] = U.a[i][j];
    }
  return C;
}
// force cross-product matrix crf(v) = -crm(v)^T
template <class T> static M6<T> crf(const T* v) {
  M6<T> C = crm(v), F;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) F.a[i][j] = -C.a[j][i];
  return F;
}
// spatial inertia about the link origin of a body with mass m, CoM c and
// rotational inertia Ic about the CoM (parallel-axis theorem):
// I = [Ic + m [c]^ [c]^T, m [c]^; m [c]^T, m 1]
static M6<double> spatial_inertia(double m, const double* c, const M3<double>& Ic) {
  M6<double> I = m6_zero<double>();
  M3<double> C = skew(c), CCt = m3_mul(C, m3_T(C));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      I.a[i][j] = Ic.a[i][j] + m * CCt.a[i][j];
      I.a[i][j + 3] = m * C.a[i][j];
      I.a[i + 3][j] = m * C.a[j][i];
    }
  for (int i = 0; i < 3; ++i) I.a[i + 3][i + 3] = m;
  return I;
}

// ---------------------------------------------------------------------------
// the evaluation
// ---------------------------------------------------------------------------
template <class T> static T joint_var(const or_robot& r, int k, const T* q) {
  return T(r.mimic_mult[k]) * q[r.jidx[k]] + T(r.mimic_off[k]);
}

static M3<double> fixed_R(const or_robot& r, int k) {
  M3<double> R;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R.a[i][j] = r.T_fixed[12 * k + 3 * i + j];
  return R;
}

// joint axis as a unit vector (the descriptor gives a direction; it is
// normalised here in double precision)
static void unit_axis(const or_robot& r, int k, double* a) {
  const double* x = r.axis + 3 * k;
  double nrm = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  for (int i = 0; i < 3; ++i) a[i] = x[i] / nrm;
}

// 1. forward kinematics: world rotation Rw[k] and origin pw[k][3]
template <class T>
static void fk(const or_robot& r, const T* q, std::vector<M3<T>>& Rw, std::vector<T>& pw) {
  Rw.resize(r.n);
  pw.assign(3 * r.n, T(0.0));
  for (int k = 0; k < r.n; ++k) {
    M3<double> Rf = fixed_R(r, k);
    const double* pf = r.T_fixed + 12 * k + 9;
    // local transform T_fixed * J(theta)
    M3<T> Rl;
    T pl[3];
    M3<T> Rft;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Rft.a[i][j] = Rf.a[i][j];
    for (int i = 0; i < 3; ++i) pl[i] = pf[i];
    double ax[3];
    unit_axis(r, k, ax);
    if (r.jtype[k] == 1) {
      Rl = m3_mul(Rft, rodrigues<T>(ax, joint_var(r, k, q)));
    } else if (r.jtype[k] == 2) {
      Rl = Rft;
      T th = joint_var(r, k, q);
      T s[3] = {T(ax[0]) * th, T(ax[1]) * th, T(ax[2]) * th};
      T Rs[3];
      m3_vec(Rft, s, Rs);
      for (int i = 0; i < 3; ++i) pl[i] = pl[i] + Rs[i];
    } else {
      Rl = Rft;
    }
    int pa = r.parent[k];
    if (pa < 0) {
      Rw[k] = Rl;
      for (int i = 0; i < 3; ++i) pw[3 * k + i] = pl[i];
    } else {
      Rw[k] = m3_mul(Rw[pa], Rl);
      T t[3];
      m3_vec(Rw[pa], pl, t);
      for (int i = 0; i < 3; ++i) pw[3 * k + i] = pw[3 * pa + i] + t[i];
    }
  }
}

// 2. sphere centres
template <class T>
static void spheres(const or_robot& r, const std::vector<M3<T>>& Rw, const std::vector<T>& pw,
                    std::vector<T>& c) {
  c.assign(3 * r.S, T(0.0));
  for (int s = 0; s < r.S; ++s) {
    int l = r.sph_link[s];
    T cl[3] = {T(r.sph_c[3 * s]), T(r.sph_c[3 * s + 1]), T(r.sph_c[3 * s + 2])};
    T t[3];
    m3_vec(Rw[l], cl, t);
    for (int i = 0; i < 3; ++i) c[3 * s + i] = t[i] + pw[3 * l + i];
  }
}

template <class T> static T pair_distance(const or_robot& r, const std::vector<T>& c, int p) {
  int i = r.pairs[2 * p], j = r.pairs[2 * p + 1];
  T dx = c[3 * i] - c[3 * j], dy = c[3 * i + 1] - c[3 * j + 1], dz = c[3 * i + 2] - c[3 * j + 2];
  return sqrt(dx * dx + dy * dy + dz * dz) - T(r.sph_r[i] + r.sph_r[j]);
}

// 3. brute-force self-collision over all masked pairs
static void self_collision(const or_robot& r, const std::vector<double>& c, double* dmin,
                           int* worst, unsigned char* collide) {
  double best = std::numeric_limits<double>::infinity();
  int bi = -1;
  for (int p = 0; p < r.P; ++p) {
    double d = pair_distance(r, c, p);
    if (collide) collide[p] = (d < 0.0) ? 1 : 0;
    if (d < best) {  // strict: the smallest index wins ties
      best = d;
      bi = p;
    }
  }
  *dmin = best;
  *worst = bi;
}

// 4. RNEA with 6x6 spatial algebra, link coordinates
template <class T>
static void rnea(const or_robot& r, const T* q, const T* qd, const T* qdd, const double* fext,
                 T* tau) {
  const int n = r.n;
  std::vector<M6<T>> X(n);
  std::vector<T> S(6 * n, T(0.0)), v(6 * n, T(0.0)), a(6 * n, T(0.0)), f(6 * n, T(0.0));
  std::vector<T> qdk(n, T(0.0)), qddk(n, T(0.0));
  for (int j = 0; j < r.d; ++j) tau[j] = T(0.0);
  for (int k = 0; k < n; ++k) {
    // X_T from the fixed transform, X_J from the joint
    M3<double> Rf = fixed_R(r, k);
    M3<T> Et;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Et.a[i][j] = Rf.a[j][i];
    T pf[3] = {T(r.T_fixed[12 * k + 9]), T(r.T_fixed[12 * k + 10]), T(r.T_fixed[12 * k + 11])};
    M6<T> XT = plucker(Et, pf);
    M6<T> XJ;
    T zero3[3] = {T(0.0), T(0.0), T(0.0)};
    double ax[3];
    unit_axis(r, k, ax);
    if (r.jtype[k] == 1) {
      T th = joint_var(r, k, q);
      XJ = plucker(m3_T(rodrigues<T>(ax, th)), zero3);
      for (int i = 0; i < 3; ++i) S[6 * k + i] = T(ax[i]);
    } else if (r.jtype[k] == 2) {
      T th = joint_var(r, k, q);
      T rr[3] = {T(ax[0]) * th, T(ax[1]) * th, T(ax[2]) * th};
      XJ = plucker(m3_eye<T>(), rr);
      for (int i = 0; i < 3; ++i) S[6 * k + 3 + i] = T(ax[i]);
    } else {
      XJ = plucker(m3_eye<T>(), zero3);
    }
    X[k] = m6_mul(XJ, XT);
    if (r.jtype[k] != 0) {
      qdk[k] = T(r.mimic_mult[k]) * qd[r.jidx[k]];
      qddk[k] = T(r.mimic_mult[k]) * qdd[r.jidx[k]];
    }
  }
  // pass 1: velocities and accelerations, base -> tips (index order)
  T abase[6] = {T(0.0), T(0.0), T(0.0), T(-r.gravity[0]), T(-r.gravity[1]), T(-r.gravity[2])};
  T vzero[6] = {T(0.0), T(0.0), T(0.0), T(0.0), T(0.0), T(0.0)};
  for (int k = 0; k < n; ++k) {
    int pa = r.parent[k];
    const T* vp = pa < 0 ? vzero : &v[6 * pa];
    const T* ap = pa < 0 ? abase : &a[6 * pa];
    T Xv[6], Xa[6];
    m6_vec(X[k], vp, Xv);
    m6_vec(X[k], ap, Xa);
    T vJ[6], c[6];
    for (int i = 0; i < 6; ++i) {
      vJ[i] = S[6 * k + i] * qdk[k];
      v[6 * k + i] = Xv[i] + vJ[i];
    }
    M6<T> cv = crm(&v[6 * k]);
    m6_vec(cv, vJ, c);
    for (int i = 0; i < 6; ++i) a[6 * k + i] = Xa[i] + S[6 * k + i] * qddk[k] + c[i];
  }
  // pass 2: per-link force f = I a + v x* I v - f_ext
  for (int k = 0; k < n; ++k) {
    M3<double> Ic;
    const double* ic = r.Icom + 6 * k;
    Ic.a[0][0] = ic[0]; Ic.a[1][1] = ic[1]; Ic.a[2][2] = ic[2];
    Ic.a[0][1] = Ic.a[1][0] = ic[3];
    Ic.a[0][2] = Ic.a[2][0] = ic[4];
    Ic.a[1][2] = Ic.a[2][1] = ic[5];
    M6<double> Id = spatial_inertia(r.mass[k], r.com + 3 * k, Ic);
    M3<double> Z;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Z.a[i][j] = 0.0;
    for (int m = 0; m < r.n_pm; ++m)
      if (r.pm_link[m] == k) {
        M6<double> Ip = spatial_inertia(r.pm_mass[m], r.pm_pos + 3 * m, Z);
        for (int i = 0; i < 6; ++i)
          for (int j = 0; j < 6; ++j) Id.a[i][j] += Ip.a[i][j];
      }
    M6<T> I;
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) I.a[i][j] = Id.a[i][j];
    T Ia[6], Iv[6], vxIv[6];
    m6_vec(I, &a[6 * k], Ia);
    m6_vec(I, &v[6 * k], Iv);
    m6_vec(crf(&v[6 * k]), Iv, vxIv);
    for (int i = 0; i < 6; ++i) {
      f[6 * k + i] = Ia[i] + vxIv[i];
      if (fext) f[6 * k + i] = f[6 * k + i] - T(fext[6 * k + i]);
    }
  }
  // pass 3: tips -> base (reverse index order), tau_j += m S^T f, f_pa += X^T f
  for (int k = n - 1; k >= 0; --k) {
    if (r.jtype[k] != 0) {
      T s = 0.0;
      for (int i = 0; i < 6; ++i) s += S[6 * k + i] * f[6 * k + i];
      tau[r.jidx[k]] += T(r.mimic_mult[k]) * s;
    }
    int pa = r.parent[k];
    if (pa >= 0) {
      T XtF[6];
      m6T_vec(X[k], &f[6 * k], XtF);
      for (int i = 0; i < 6; ++i) f[6 * pa + i] += XtF[i];
    }
  }
}

// scalar loss for the gradient: <gpose,pose> + <gsph,c> + gdmin*d_worst + <gtau,tau>
template <class T>
static T loss(const or_robot& r, const T* q, const T* qd, const T* qdd, const double* fext,
              int worst, const double* gpose, const double* gsph, double gdmin,
              const double* gtau) {
  std::vector<M3<T>> Rw;
  std::vector<T> pw, c;
  fk(r, q, Rw, pw);
  T L = 0.0;
  if (gpose)
    for (int k = 0; k < r.n; ++k) {
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) L += T(gpose[12 * k + 3 * i + j]) * Rw[k].a[i][j];
      for (int i = 0; i < 3; ++i) L += T(gpose[12 * k + 9 + i]) * pw[3 * k + i];
    }
  if (gsph || (gdmin != 0.0 && worst >= 0)) {
    spheres(r, Rw, pw, c);
    if (gsph)
      for (int s = 0; s < 3 * r.S; ++s) L += T(gsph[s]) * c[s];
    if (gdmin != 0.0 && worst >= 0) L += T(gdmin) * pair_distance(r, c, worst);
  }
  if (gtau) {
    std::vector<T> tau(r.d);
    rnea(r, q, qd, qdd, fext, tau.data());
    for (int j = 0; j < r.d; ++j) L += T(gtau[j]) * tau[j];
  }
  return L;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
static int threads_for(int nthreads) {
#ifdef _OPENMP
  return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

extern "C" {

int or_version(void) { return 1; }

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// Forward evaluation of B configurations.  All arrays config-major:
// q, qd, qdd, tau [B][d]; pose [B][n][12]; sph [B][S][3]; dmin [B]; worst [B];
// collide [B][P]; fext [B][n][6] (link-frame spatial force, nullable).
// Any output may be NULL to skip it.
int or_eval(const or_robot* r, int B, const double* q, const double* qd, const double* qdd,
            const double* fext, double* pose, double* sph, double* dmin, int* worst,
            unsigned char* collide, double* tau, int nthreads) {
  int nt = threads_for(nthreads);
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
  for (int b = 0; b < B; ++b) {
    const double* qb = q + (size_t)b * r->d;
    std::vector<M3<double>> Rw;
    std::vector<double> pw, c;
    fk(*r, qb, Rw, pw);
    if (pose)
      for (int k = 0; k < r->n; ++k) {
        double* o = pose + ((size_t)b * r->n + k) * 12;
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) o[3 * i + j] = Rw[k].a[i][j];
        for (int i = 0; i < 3; ++i) o[9 + i] = pw[3 * k + i];
      }
    spheres(*r, Rw, pw, c);
    if (sph) std::memcpy(sph + (size_t)b * r->S * 3, c.data(), sizeof(double) * 3 * r->S);
    if (dmin || worst || collide) {
      double dm;
      int w;
      self_collision(*r, c, &dm, &w, collide ? collide + (size_t)b * r->P : nullptr);
      if (dmin) dmin[b] = dm;
      if (worst) worst[b] = w;
    }
    if (tau)
      rnea(*r, qb, qd + (size_t)b * r->d, qdd + (size_t)b * r->d,
           fext ? fext + (size_t)b * r->n * 6 : nullptr, tau + (size_t)b * r->d);
  }
  return 0;
}

// Gradient of L (see loss) for B configurations.  gpose [B][n][12],
// gsph [B][S][3], gdmin [B], gtau [B][d] (each nullable = zero);
// outputs gq, gqd, gqdd [B][d].  The worst pair is found in double first and
// the dual passes differentiate through that pair.
int or_grad(const or_robot* r, int B, const double* q, const double* qd, const double* qdd,
            const double* fext, const double* gpose, const double* gsph, const double* gdmin,
            const double* gtau, double* gq, double* gqd, double* gqdd, int nthreads) {
  int nt = threads_for(nthreads);
  const int d = r->d;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
  for (int b = 0; b < B; ++b) {
    const double* qb = q + (size_t)b * d;
    const double* qdb = qd + (size_t)b * d;
    const double* qddb = qdd + (size_t)b * d;
    double gdm = gdmin ? gdmin[b] : 0.0;
    int worst = -1;
    if (gdm != 0.0) {
      std::vector<M3<double>> Rw;
      std::vector<double> pw, c;
      fk(*r, qb, Rw, pw);
      spheres(*r, Rw, pw, c);
      double dm;
      self_collision(*r, c, &dm, &worst, nullptr);
    }
    const double* gp = gpose ? gpose + (size_t)b * r->n * 12 : nullptr;
    const double* gs = gsph ? gsph + (size_t)b * r->S * 3 : nullptr;
    const double* gt = gtau ? gtau + (size_t)b * d : nullptr;
    const double* fe = fext ? fext + (size_t)b * r->n * 6 : nullptr;
    std::vector<Dual> Q(d), QD(d), QDD(d);
    for (int which = 0; which < 3; ++which)
      for (int j = 0; j < d; ++j) {
        for (int i = 0; i < d; ++i) {
          Q[i] = Dual(qb[i], (which == 0 && i == j) ? 1.0 : 0.0);
          QD[i] = Dual(qdb[i], (which == 1 && i == j) ? 1.0 : 0.0);
          QDD[i] = Dual(qddb[i], (which == 2 && i == j) ? 1.0 : 0.0);
        }
        // q-independent terms are skipped for the qd / qdd directions
        const double* gp_ = which == 0 ? gp : nullptr;
        const double* gs_ = which == 0 ? gs : nullptr;
        double gdm_ = which == 0 ? gdm : 0.0;
        Dual L = loss(*r, Q.data(), QD.data(), QDD.data(), fe, worst, gp_, gs_, gdm_, gt);
        double* out = which == 0 ? gq : (which == 1 ? gqd : gqdd);
        out[(size_t)b * d + j] = L.d;
      }
  }
  return 0;
}

// L (see loss) from one full forward evaluation in double: FK, sphere
// centres, the brute-force minimum over every masked pair and the RNEA
// torques, as or_eval computes them.
static double full_loss(const or_robot& r, const double* q, const double* qd, const double* qdd,
                        const double* fext, const double* gpose, const double* gsph,
                        double gdmin, const double* gtau) {
  std::vector<M3<double>> Rw;
  std::vector<double> pw, c, tau(r.d);
  fk(r, q, Rw, pw);
  spheres(r, Rw, pw, c);
  double dm = 0.0;
  int w = -1;
  self_collision(r, c, &dm, &w, nullptr);
  rnea(r, q, qd, qdd, fext, tau.data());
  double L = 0.0;
  if (gpose)
    for (int k = 0; k < r.n; ++k) {
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) L += gpose[12 * k + 3 * i + j] * Rw[k].a[i][j];
      for (int i = 0; i < 3; ++i) L += gpose[12 * k + 9 + i] * pw[3 * k + i];
    }
  if (gsph)
    for (int s = 0; s < 3 * r.S; ++s) L += gsph[s] * c[s];
  if (gdmin != 0.0 && w >= 0) L += gdmin * dm;
  if (gtau)
    for (int j = 0; j < r.d; ++j) L += gtau[j] * tau[j];
  return L;
}

// The same gradient as or_grad by central differences of full forward
// evaluations: two at x +- h e_i for each of the 3d inputs per configuration
// (with the forward evaluation at the point itself, 2*3d + 1 evaluations:
// the gradient a CPU program without an adjoint would compute).  d_min
// enters as the minimum over all pairs, so the difference is valid where no
// other pair takes over the minimum within +-h.  Outputs gq, gqd, gqdd [B][d].
int or_grad_fd(const or_robot* r, int B, const double* q, const double* qd, const double* qdd,
               const double* fext, const double* gpose, const double* gsph, const double* gdmin,
               const double* gtau, double h, double* gq, double* gqd, double* gqdd,
               int nthreads) {
  if (!(h > 0.0)) return -1;
  int nt = threads_for(nthreads);
  const int d = r->d;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
  for (int b = 0; b < B; ++b) {
    std::vector<double> x[3] = {std::vector<double>(q + (size_t)b * d, q + (size_t)(b + 1) * d),
                                std::vector<double>(qd + (size_t)b * d, qd + (size_t)(b + 1) * d),
                                std::vector<double>(qdd + (size_t)b * d,
                                                    qdd + (size_t)(b + 1) * d)};
    const double* gp = gpose ? gpose + (size_t)b * r->n * 12 : nullptr;
    const double* gs = gsph ? gsph + (size_t)b * r->S * 3 : nullptr;
    const double gdm = gdmin ? gdmin[b] : 0.0;
    const double* gt = gtau ? gtau + (size_t)b * d : nullptr;
    const double* fe = fext ? fext + (size_t)b * r->n * 6 : nullptr;
    auto L = [&]() {
      return full_loss(*r, x[0].data(), x[1].data(), x[2].data(), fe, gp, gs, gdm, gt);
    };
    double* out[3] = {gq, gqd, gqdd};
    for (int which = 0; which < 3; ++which)
      for (int j = 0; j < d; ++j) {
        const double x0 = x[which][j];
        x[which][j] = x0 + h;
        const double lp = L();
        x[which][j] = x0 - h;
        const double lm = L();
        x[which][j] = x0;
        out[which][(size_t)b * d + j] = (lp - lm) / (2.0 * h);
      }
  }
  return 0;
}

// Uniform cubic B-spline (Sec. 4, Eq. bspline-cubic).  U [n_traj][d][K]
// control points; each trajectory is sampled at T uniformly spaced points over
// its K-3 valid segments: t_s = s*(K-3)/(T-1), segment k = min(floor(t_s), K-4),
// alpha = t_s - k, local control vector [u_k, u_k+1, u_k+2, u_k+3].
// Outputs q, qd, qdd [n_traj*T][d] (config b = traj*T + s).
int or_bspline(int n_traj, int d, int K, int T, double dt, const double* U, double* q,
               double* qd, double* qdd) {
  if (K < 4 || T < 2) return -1;
  const double C[4][4] = {{-1.0 / 6, 3.0 / 6, -3.0 / 6, 1.0 / 6},
                          {3.0 / 6, -6.0 / 6, 3.0 / 6, 0.0},
                          {-3.0 / 6, 0.0, 3.0 / 6, 0.0},
                          {1.0 / 6, 4.0 / 6, 1.0 / 6, 0.0}};
  const int nseg = K - 3;
  for (int tr = 0; tr < n_traj; ++tr)
    for (int s = 0; s < T; ++s) {
      double t = (double)s * nseg / (double)(T - 1);
      int k = (int)std::floor(t);
      if (k > nseg - 1) k = nseg - 1;
      double al = t - k;
      // rows of T P(alpha)
      double P[3][4] = {{al * al * al, al * al, al, 1.0},
                        {3 * al * al / dt, 2 * al / dt, 1.0 / dt, 0.0},
                        {6 * al / (dt * dt), 2.0 / (dt * dt), 0.0, 0.0}};
      for (int j = 0; j < d; ++j) {
        const double* u = U + ((size_t)tr * d + j) * K + k;
        double out[3];
        for (int row = 0; row < 3; ++row) {
          double acc = 0.0;
          for (int m = 0; m < 4; ++m) {
            double cu = 0.0;
            for (int l = 0; l < 4; ++l) cu += C[m][l] * u[l];
            acc += P[row][m] * cu;
          }
          out[row] = acc;
        }
        size_t b = (size_t)tr * T + s;
        q[b * d + j] = out[0];
        qd[b * d + j] = out[1];
        qdd[b * d + j] = out[2];
      }
    }
  return 0;
}

// Kinematic Jacobians and the centre of mass (Sec. 6.1.1 "centers of mass,
// and Jacobians"; Alg. 2 gives their column structure), by forward-mode
// differentiation of the forward kinematics: one dual pass per joint j seeds
// dq_j = 1.  For target link e, column j of J [B][nt][6][d] holds the
// derivative of e's world origin (rows 0-2) and the angular velocity of its
// frame, vee(dR_e/dq_j R_e^T) (rows 3-5).  com [B][3] is the mass-weighted mean
// of the link centres of mass and the payload point masses; Jcom [B][3][d] its
// derivative.  Each output may be NULL.
int or_kinematics(const or_robot* r, int B, const double* q, int nt, const int* targets,
                  double* J, double* com, double* Jcom, int nthreads) {
  const int d = r->d, n = r->n;
  for (int t = 0; t < nt; ++t)
    if (targets[t] < 0 || targets[t] >= n) return -1;
  double M = 0.0;
  for (int k = 0; k < n; ++k) M += r->mass[k];
  for (int m = 0; m < r->n_pm; ++m) M += r->pm_mass[m];
  int nthr = threads_for(nthreads);
#pragma omp parallel for num_threads(nthr) schedule(dynamic, 1)
  for (int b = 0; b < B; ++b) {
    const double* qb = q + (size_t)b * d;
    // centre of mass of the configuration, with derivative along seed j
    auto com_of = [&](const std::vector<M3<Dual>>& Rw, const std::vector<Dual>& pw, Dual* c) {
      c[0] = c[1] = c[2] = Dual(0.0);
      auto add_point = [&](int k, const double* x, double m) {
        Dual cl[3] = {Dual(x[0]), Dual(x[1]), Dual(x[2])}, wc[3];
        m3_vec(Rw[k], cl, wc);
        for (int i = 0; i < 3; ++i) c[i] += Dual(m) * (wc[i] + pw[3 * k + i]);
      };
      for (int k = 0; k < n; ++k) add_point(k, r->com + 3 * k, r->mass[k]);
      for (int m = 0; m < r->n_pm; ++m) add_point(r->pm_link[m], r->pm_pos + 3 * m, r->pm_mass[m]);
      for (int i = 0; i < 3; ++i) c[i] = c[i] / Dual(M);
    };
    for (int j = 0; j < std::max(d, 1); ++j) {
      std::vector<Dual> qd(d);
      for (int i = 0; i < d; ++i) qd[i] = Dual(qb[i], i == j ? 1.0 : 0.0);
      std::vector<M3<Dual>> Rw;
      std::vector<Dual> pw;
      fk(*r, qd.data(), Rw, pw);
      if (d == 0) break;
      for (int t = 0; t < nt; ++t) {
        const int e = targets[t];
        double* col = J ? J + (((size_t)b * nt + t) * 6) * d + j : nullptr;
        if (!col) break;
        for (int i = 0; i < 3; ++i) col[(size_t)i * d] = pw[3 * e + i].d;
        // W = dR R^T is skew; its axial vector is the angular velocity
        double Wm[3][3];
        for (int i = 0; i < 3; ++i)
          for (int k = 0; k < 3; ++k) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l) acc += Rw[e].a[i][l].d * Rw[e].a[k][l].v;
            Wm[i][k] = acc;
          }
        col[3 * (size_t)d] = 0.5 * (Wm[2][1] - Wm[1][2]);
        col[4 * (size_t)d] = 0.5 * (Wm[0][2] - Wm[2][0]);
        col[5 * (size_t)d] = 0.5 * (Wm[1][0] - Wm[0][1]);
      }
      if (com || Jcom) {
        Dual c[3];
        com_of(Rw, pw, c);
        if (com && j == 0)
          for (int i = 0; i < 3; ++i) com[3 * (size_t)b + i] = c[i].v;
        if (Jcom)
          for (int i = 0; i < 3; ++i) Jcom[((size_t)b * 3 + i) * d + j] = c[i].d;
      }
    }
  }
  return 0;
}

// Vector-Jacobian product of or_bspline (Eq. backward_grad): every sample adds
// B(alpha)^T g to the four control points of its window, B = T P(alpha) C with
// the rows for theta, theta_dot, theta_ddot.  gq, gqd, gqdd [n_traj*T][d]
// (each may be NULL = zero); Ubar [n_traj][d][K] is overwritten.
int or_bspline_vjp(int n_traj, int d, int K, int T, double dt, const double* gq,
                   const double* gqd, const double* gqdd, double* Ubar) {
  if (K < 4 || T < 2) return -1;
  const double C[4][4] = {{-1.0 / 6, 3.0 / 6, -3.0 / 6, 1.0 / 6},
                          {3.0 / 6, -6.0 / 6, 3.0 / 6, 0.0},
                          {-3.0 / 6, 0.0, 3.0 / 6, 0.0},
                          {1.0 / 6, 4.0 / 6, 1.0 / 6, 0.0}};
  const int nseg = K - 3;
  std::fill(Ubar, Ubar + (size_t)n_traj * d * K, 0.0);
  for (int tr = 0; tr < n_traj; ++tr)
    for (int s = 0; s < T; ++s) {
      double t = (double)s * nseg / (double)(T - 1);
      int k = (int)std::floor(t);
      if (k > nseg - 1) k = nseg - 1;
      double al = t - k;
      double P[3][4] = {{al * al * al, al * al, al, 1.0},
                        {3 * al * al / dt, 2 * al / dt, 1.0 / dt, 0.0},
                        {6 * al / (dt * dt), 2.0 / (dt * dt), 0.0, 0.0}};
      double Bm[3][4];
      for (int row = 0; row < 3; ++row)
        for (int l = 0; l < 4; ++l) {
          double acc = 0.0;
          for (int m = 0; m < 4; ++m) acc += P[row][m] * C[m][l];
          Bm[row][l] = acc;
        }
      const size_t b = (size_t)tr * T + s;
      for (int j = 0; j < d; ++j) {
        const double g[3] = {gq ? gq[b * d + j] : 0.0, gqd ? gqd[b * d + j] : 0.0,
                             gqdd ? gqdd[b * d + j] : 0.0};
        double* u = Ubar + ((size_t)tr * d + j) * K + k;
        for (int l = 0; l < 4; ++l)
          u[l] += Bm[0][l] * g[0] + Bm[1][l] * g[1] + Bm[2][l] * g[2];
      }
    }
  return 0;
}

}  // extern "C"
