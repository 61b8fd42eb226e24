// FP64 CPU oracle for the multiple-shooting SVGD hot path.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may load, call or
// link this file: only the test suite, the smoke check and the benchmark's
// CPU-baseline leg use it.  It shares no code, header or constant with the
// CUDA library; its only common ground with that library is the seeded input
// generator, which holds none of the method's arithmetic.
//
// Everything here is plain, slow and double precision, written to be checked
// against the paper by eye:
//   * planar articulated-body forward dynamics (ABA, Featherstone's
//     articulated-body recursion in link-local Plucker frames), the step of
//     Appendix B-A, Eq. (dynamics);
//   * CRBA + Cholesky, a second forward-dynamics algorithm used only as a
//     cross-check of the ABA;
//   * semi-implicit Euler exactly as Eq. (dynamics): acceleration, then
//     velocity, then position with the new velocity;
//   * the multiple-shooting log-likelihood of Sec. IV-C (Eqs. 2, 4, 5) plus
//     the parameter-limit prior of Sec. IV-D;
//   * its gradient by forward-mode dual numbers, one window at a time
//     (exact up to rounding, independent of the GPU's reverse adjoint);
//   * the SVGD update of Eq. (1) with an RBF kernel and the median heuristic
//     (Sec. IV-A), driven by Adam (Algorithm 1's "learning rate scheduler");
//   * constrained SVGD (Sec. IV-E, Algorithm 1): the observation likelihood,
//     the defect and limit constraints, their MDMM gradient with the
//     per-particle multipliers held fixed, and the MDMM update.
//
// Readings taken where the paper is silent (the GPU path takes the same ones):
//   window w covers steps t_w+1 .. t_{w+1}, t_w = floor(w*T/W); window 0
//   starts at the known s_0, window w>0 at the shooting state s^s_w; every
//   observation x_1..x_T is compared once; Gaussian constants are included;
//   the uniform limit prior is log U = -sum log(hi-lo) plus the smooth
//   penalty -(c_lim/2)||clamp(u,0,1)-u||^2 in the unit box u; the kernel acts
//   on the unit-box coordinates u of theta; bandwidth = lower median of the
//   pairwise squared distances over i<j divided by log N.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// ---------------------------------------------------------------------------
// Forward-mode dual numbers (value + up to MAXD directional derivatives).
// The number of live directions is a per-thread setting.
// ---------------------------------------------------------------------------
constexpr int MAXD = 72;
static thread_local int g_nd = 0;

struct Dual {
  double v;
  double d[MAXD];
  Dual() : v(0.0) { std::memset(d, 0, sizeof(d)); }
  Dual(double x) : v(x) { std::memset(d, 0, sizeof(d)); }
};
static inline Dual operator+(const Dual& a, const Dual& b) {
  Dual r(a.v + b.v);
  for (int k = 0; k < g_nd; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
static inline Dual operator-(const Dual& a, const Dual& b) {
  Dual r(a.v - b.v);
  for (int k = 0; k < g_nd; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
static inline Dual operator-(const Dual& a) {
  Dual r(-a.v);
  for (int k = 0; k < g_nd; ++k) r.d[k] = -a.d[k];
  return r;
}
static inline Dual operator*(const Dual& a, const Dual& b) {
  Dual r(a.v * b.v);
  for (int k = 0; k < g_nd; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
  return r;
}
static inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v);
  const double inv = 1.0 / b.v;
  for (int k = 0; k < g_nd; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * inv;
  return r;
}
static inline Dual& operator+=(Dual& a, const Dual& b) { a = a + b; return a; }
static inline Dual& operator-=(Dual& a, const Dual& b) { a = a - b; return a; }
static inline Dual sin(const Dual& a) {
  Dual r(std::sin(a.v));
  const double c = std::cos(a.v);
  for (int k = 0; k < g_nd; ++k) r.d[k] = c * a.d[k];
  return r;
}
static inline Dual cos(const Dual& a) {
  Dual r(std::cos(a.v));
  const double s = -std::sin(a.v);
  for (int k = 0; k < g_nd; ++k) r.d[k] = s * a.d[k];
  return r;
}
static inline double val(double x) { return x; }
static inline double val(const Dual& x) { return x.v; }
using std::sin;
using std::cos;

// ---------------------------------------------------------------------------
// Planar spatial algebra (3-vectors (omega, vx, vy) / (n, fx, fy)).
// ---------------------------------------------------------------------------
template <class T> struct V3 { T a[3]; };
template <class T> struct M3 { T a[3][3]; };

template <class T> static V3<T> vzero() { V3<T> r; for (int i = 0; i < 3; ++i) r.a[i] = T(0.0); return r; }
template <class T> static M3<T> mzero() { M3<T> r; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) r.a[i][j] = T(0.0); return r; }

template <class T> static V3<T> mul(const M3<T>& m, const V3<T>& v) {
  V3<T> r;
  for (int i = 0; i < 3; ++i) r.a[i] = m.a[i][0] * v.a[0] + m.a[i][1] * v.a[1] + m.a[i][2] * v.a[2];
  return r;
}
template <class T> static V3<T> mulT(const M3<T>& m, const V3<T>& v) {  // m^T v
  V3<T> r;
  for (int i = 0; i < 3; ++i) r.a[i] = m.a[0][i] * v.a[0] + m.a[1][i] * v.a[1] + m.a[2][i] * v.a[2];
  return r;
}
template <class T> static M3<T> mul(const M3<T>& x, const M3<T>& y) {
  M3<T> r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.a[i][j] = x.a[i][0] * y.a[0][j] + x.a[i][1] * y.a[1][j] + x.a[i][2] * y.a[2][j];
  return r;
}
template <class T> static M3<T> transpose(const M3<T>& x) {
  M3<T> r;
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) r.a[i][j] = x.a[j][i];
  return r;
}
template <class T> static V3<T> add(const V3<T>& x, const V3<T>& y) { V3<T> r; for (int i = 0; i < 3; ++i) r.a[i] = x.a[i] + y.a[i]; return r; }
template <class T> static V3<T> sub(const V3<T>& x, const V3<T>& y) { V3<T> r; for (int i = 0; i < 3; ++i) r.a[i] = x.a[i] - y.a[i]; return r; }
template <class T> static M3<T> add(const M3<T>& x, const M3<T>& y) { M3<T> r; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) r.a[i][j] = x.a[i][j] + y.a[i][j]; return r; }

// Plucker transform of motion vectors from frame A to frame B, where B's
// origin sits at r (A coordinates) and B is rotated by th relative to A.
template <class T> static M3<T> plnr(const T& th, const T& rx, const T& ry) {
  T c = cos(th), s = sin(th);
  M3<T> X;
  X.a[0][0] = T(1.0); X.a[0][1] = T(0.0); X.a[0][2] = T(0.0);
  X.a[1][0] = s * rx - c * ry; X.a[1][1] = c; X.a[1][2] = s;
  X.a[2][0] = c * rx + s * ry; X.a[2][1] = -s; X.a[2][2] = c;
  return X;
}
// motion cross product v x m
template <class T> static V3<T> crm(const V3<T>& v, const V3<T>& m) {
  V3<T> r;
  r.a[0] = T(0.0);
  r.a[1] = v.a[2] * m.a[0] - v.a[0] * m.a[2];
  r.a[2] = v.a[0] * m.a[1] - v.a[1] * m.a[0];
  return r;
}
// force cross product v x* f
template <class T> static V3<T> crf(const V3<T>& v, const V3<T>& f) {
  V3<T> r;
  r.a[0] = v.a[1] * f.a[2] - v.a[2] * f.a[1];
  r.a[1] = -v.a[0] * f.a[2];
  r.a[2] = v.a[0] * f.a[1];
  return r;
}
// Planar spatial inertia of a point mass m at (cx, cy) in the link frame.
template <class T> static M3<T> point_inertia(const T& m, const T& cx, const T& cy) {
  M3<T> I;
  I.a[0][0] = m * (cx * cx + cy * cy); I.a[0][1] = -(m * cy); I.a[0][2] = m * cx;
  I.a[1][0] = -(m * cy);               I.a[1][1] = m;         I.a[1][2] = T(0.0);
  I.a[2][0] = m * cx;                  I.a[2][1] = T(0.0);    I.a[2][2] = m;
  return I;
}

// ---------------------------------------------------------------------------
// Planar serial chain of revolute joints, point mass m_i at the tip of link i,
// relative joint angles, q = 0 hanging straight down, gravity -g y.
// Joint torque is viscous damping tau_i = -b_i qd_i (no actuation).
// Link frame i: origin at joint i, rotated by the absolute link angle; the
// link runs along its local -y axis, so its tip (and mass) is at (0, -l_i).
// ---------------------------------------------------------------------------
template <class T> struct Chain {
  int n;
  const T* m;
  const T* l;
  const T* b;
  double g;
};

template <class T> static M3<T> joint_xup(const Chain<T>& ch, int i, const T& qi) {
  // Joint i sits at the tip of link i-1, i.e. at (0, -l_{i-1}) in frame i-1.
  if (i == 0) return plnr<T>(qi, T(0.0), T(0.0));
  return plnr<T>(qi, T(0.0), -ch.l[i - 1]);
}

// Articulated-body algorithm (three passes: velocities outward, articulated
// inertias inward, accelerations outward).  Appendix B-A names ABA as the
// forward dynamics inside f_step.
template <class T>
static void aba(const Chain<T>& ch, const T* q, const T* qd, const T* tau, T* qdd) {
  const int n = ch.n;
  std::vector<M3<T>> Xup(n), IA(n);
  std::vector<V3<T>> v(n), c(n), pA(n), U(n), a(n);
  std::vector<T> d(n), u(n);
  for (int i = 0; i < n; ++i) {
    Xup[i] = joint_xup(ch, i, q[i]);
    V3<T> vJ = vzero<T>();
    vJ.a[0] = qd[i];
    v[i] = (i == 0) ? vJ : add(mul(Xup[i], v[i - 1]), vJ);
    c[i] = crm(v[i], vJ);
    M3<T> I = point_inertia<T>(ch.m[i], T(0.0), -ch.l[i]);
    IA[i] = I;
    pA[i] = crf(v[i], mul(I, v[i]));
  }
  for (int i = n - 1; i >= 0; --i) {
    U[i].a[0] = IA[i].a[0][0]; U[i].a[1] = IA[i].a[1][0]; U[i].a[2] = IA[i].a[2][0];
    d[i] = U[i].a[0];
    u[i] = tau[i] - pA[i].a[0];
    if (i > 0) {
      M3<T> Ia;
      for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) Ia.a[r][s] = IA[i].a[r][s] - U[i].a[r] * U[i].a[s] / d[i];
      V3<T> pa = mul(Ia, c[i]);
      for (int r = 0; r < 3; ++r) pa.a[r] = pA[i].a[r] + pa.a[r] + U[i].a[r] * u[i] / d[i];
      IA[i - 1] = add(IA[i - 1], mul(transpose(Xup[i]), mul(Ia, Xup[i])));
      pA[i - 1] = add(pA[i - 1], mulT(Xup[i], pa));
    }
  }
  V3<T> a0 = vzero<T>();
  a0.a[2] = T(ch.g);  // fictitious base acceleration = -gravity
  for (int i = 0; i < n; ++i) {
    a[i] = add(mul(Xup[i], (i == 0) ? a0 : a[i - 1]), c[i]);
    qdd[i] = (u[i] - (U[i].a[0] * a[i].a[0] + U[i].a[1] * a[i].a[1] + U[i].a[2] * a[i].a[2])) / d[i];
    a[i].a[0] = a[i].a[0] + qdd[i];
  }
}

// Composite-rigid-body algorithm + recursive Newton-Euler bias; used only to
// cross-check the ABA.  H qdd = tau - C.
static void crba_bias(const Chain<double>& ch, const double* q, const double* qd, double* H, double* C) {
  const int n = ch.n;
  std::vector<M3<double>> Xup(n), IC(n), I(n);
  std::vector<V3<double>> v(n), a(n), f(n);
  for (int i = 0; i < n; ++i) {
    Xup[i] = joint_xup(ch, i, q[i]);
    I[i] = point_inertia<double>(ch.m[i], 0.0, -ch.l[i]);
    V3<double> vJ = vzero<double>();
    vJ.a[0] = qd[i];
    V3<double> a0 = vzero<double>();
    a0.a[2] = ch.g;
    v[i] = (i == 0) ? vJ : add(mul(Xup[i], v[i - 1]), vJ);
    a[i] = add(mul(Xup[i], (i == 0) ? a0 : a[i - 1]), crm(v[i], vJ));
    f[i] = add(mul(I[i], a[i]), crf(v[i], mul(I[i], v[i])));
    IC[i] = I[i];
  }
  for (int i = n - 1; i >= 0; --i) {
    C[i] = f[i].a[0];
    if (i > 0) {
      f[i - 1] = add(f[i - 1], mulT(Xup[i], f[i]));
      IC[i - 1] = add(IC[i - 1], mul(transpose(Xup[i]), mul(IC[i], Xup[i])));
    }
  }
  for (int i = 0; i < n; ++i) {
    V3<double> F;
    F.a[0] = IC[i].a[0][0]; F.a[1] = IC[i].a[1][0]; F.a[2] = IC[i].a[2][0];
    H[i * n + i] = F.a[0];
    int j = i;
    while (j > 0) {
      F = mulT(Xup[j], F);
      --j;
      H[i * n + j] = F.a[0];
      H[j * n + i] = F.a[0];
    }
  }
}

static bool cholesky_solve(int n, const double* H, const double* rhs, double* x) {
  std::vector<double> L(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = H[i * n + j];
      for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
      if (i == j) {
        if (s <= 0.0) return false;
        L[i * n + i] = std::sqrt(s);
      } else {
        L[i * n + j] = s / L[j * n + j];
      }
    }
  }
  std::vector<double> y(n);
  for (int i = 0; i < n; ++i) {
    double s = rhs[i];
    for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
    y[i] = s / L[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
  return true;
}

// One semi-implicit Euler step, Eq. (dynamics): qdd from (q_t, qd_t), then
// qd_{t+1} = qd_t + qdd dt, then q_{t+1} = q_t + qd_{t+1} dt.
// State layout s = [q_0..q_{n-1}, qd_0..qd_{n-1}].
template <class T>
static void step(const Chain<T>& ch, double dt, const T* s, T* s_next) {
  const int n = ch.n;
  std::vector<T> tau(n), qdd(n);
  for (int i = 0; i < n; ++i) tau[i] = -(ch.b[i] * s[n + i]);
  aba(ch, s, s + n, tau.data(), qdd.data());
  for (int i = 0; i < n; ++i) {
    T qd_new = s[n + i] + qdd[i] * T(dt);
    s_next[n + i] = qd_new;
    s_next[i] = s[i] + qd_new * T(dt);
  }
}

// ---------------------------------------------------------------------------
// Problem description shared by the likelihood functions.
// ---------------------------------------------------------------------------
struct Problem {
  int n;                   // links
  double g;
  const double* mass;      // [n] values used where theta does not override
  const double* length;    // [n]
  const double* damping;   // [n]
  int M;                   // dim theta
  const int* theta_kind;   // [M] 0 mass, 1 length, 2 damping
  const int* theta_link;   // [M]
  double dt;
  int T, W, D;
  const int* obs_index;    // [D] indices into the state
  const double* obs;       // [T][D], row t-1 holds x_t
  double sigma_obs, sigma_def;
  const double* s0;        // [2n]
  const double* lo;        // [M]
  const double* hi;        // [M]
  double c_lim;
  // a set of R trajectories (Sec. IV-C, Eqs. traj_likelihood_sum/_prod):
  // obs is then [R][T][D] and s0 [R][2n]; each trajectory has its own
  // shooting states.  combine: 0 sum (equally weighted mixture), 1 product.
  int R;
  int combine;
};

static inline int window_start(const Problem& P, int w) { return (int)(((long long)w * P.T) / P.W); }

// log N(x | mu, sigma^2 I) for a single scalar component, without the
// constant (the constant is added once per vector below).
// The window's log-likelihood: observation terms for t = t_w+1 .. t_{w+1}
// (Eq. 2 over the window, Eq. 5's inner factor) and, for w < W-1, the
// defect term log N(s^s_{w+1} | s_end, sigma_def^2 I) (Eq. 4).
template <class T>
static T window_loglik(const Problem& P, const T* m, const T* l, const T* b, const T* s_start, const T* s_next, int w) {
  const int n = P.n, S = 2 * n;
  Chain<T> ch{n, m, l, b, P.g};
  std::vector<T> s(s_start, s_start + S), sn(S);
  const int t0 = window_start(P, w), t1 = window_start(P, w + 1);
  const double so2 = P.sigma_obs * P.sigma_obs;
  const double obs_const = -0.5 * P.D * std::log(2.0 * M_PI * so2);
  T ll(0.0);
  for (int t = t0 + 1; t <= t1; ++t) {
    step(ch, P.dt, s.data(), sn.data());
    s.swap(sn);
    T acc(0.0);
    for (int k = 0; k < P.D; ++k) {
      T r = T(P.obs[(size_t)(t - 1) * P.D + k]) - s[P.obs_index[k]];
      acc += r * r;
    }
    ll += acc * T(-0.5 / so2) + T(obs_const);
  }
  if (w < P.W - 1) {
    const double sd2 = P.sigma_def * P.sigma_def;
    T acc(0.0);
    for (int k = 0; k < S; ++k) {
      T d = s_next[k] - s[k];
      acc += d * d;
    }
    ll += acc * T(-0.5 / sd2) + T(-0.5 * S * std::log(2.0 * M_PI * sd2));
  }
  return ll;
}

// Physical link parameters for one particle: defaults overridden by theta.
template <class T>
static void physical_params(const Problem& P, const T* theta, std::vector<T>& m, std::vector<T>& l, std::vector<T>& b) {
  m.assign(P.n, T(0.0)); l.assign(P.n, T(0.0)); b.assign(P.n, T(0.0));
  for (int i = 0; i < P.n; ++i) { m[i] = T(P.mass[i]); l[i] = T(P.length[i]); b[i] = T(P.damping[i]); }
  for (int k = 0; k < P.M; ++k) {
    const int i = P.theta_link[k];
    if (P.theta_kind[k] == 0) m[i] = theta[k];
    else if (P.theta_kind[k] == 1) l[i] = theta[k];
    else b[i] = theta[k];
  }
}

// log p_lim: uniform density on the box plus the smooth limit penalty.
static double limit_logprior(const Problem& P, const double* theta, double* grad_theta) {
  double lp = 0.0;
  for (int k = 0; k < P.M; ++k) {
    const double w = P.hi[k] - P.lo[k];
    const double u = (theta[k] - P.lo[k]) / w;
    const double cu = std::min(1.0, std::max(0.0, u));
    lp += -std::log(w) - 0.5 * P.c_lim * (cu - u) * (cu - u);
    if (grad_theta) grad_theta[k] += P.c_lim * (cu - u) / w;
  }
  return lp;
}

// log p_ms for one particle (Eq. 5 summed in log space) plus log p_lim, and
// its gradient over the augmented vector [theta, s^s_1 .. s^s_{W-1}].
static double particle_loglik_grad(const Problem& P, const double* x, double* grad) {
  const int n = P.n, S = 2 * n, M = P.M, W = P.W;
  const int Pdim = M + (W - 1) * S;
  if (grad) std::fill(grad, grad + Pdim, 0.0);
  double total = 0.0;
  for (int w = 0; w < W; ++w) {
    const double* ss = (w == 0) ? P.s0 : x + M + (w - 1) * S;
    const double* sn = (w < W - 1) ? x + M + w * S : nullptr;
    if (!grad) {
      std::vector<double> m, l, b;
      physical_params<double>(P, x, m, l, b);
      total += window_loglik<double>(P, m.data(), l.data(), b.data(), ss, sn, w);
      continue;
    }
    // Directions: theta (M), start state (S, only for w>0), next state (S).
    g_nd = M + 2 * S;
    std::vector<Dual> th(M), s_start(S), s_next(S);
    for (int k = 0; k < M; ++k) { th[k] = Dual(x[k]); th[k].d[k] = 1.0; }
    for (int k = 0; k < S; ++k) {
      s_start[k] = Dual(ss[k]);
      if (w > 0) s_start[k].d[M + k] = 1.0;
      if (sn) { s_next[k] = Dual(sn[k]); s_next[k].d[M + S + k] = 1.0; }
    }
    std::vector<Dual> m, l, b;
    physical_params<Dual>(P, th.data(), m, l, b);
    Dual ll = window_loglik<Dual>(P, m.data(), l.data(), b.data(), s_start.data(), sn ? s_next.data() : nullptr, w);
    total += ll.v;
    for (int k = 0; k < M; ++k) grad[k] += ll.d[k];
    if (w > 0)
      for (int k = 0; k < S; ++k) grad[M + (w - 1) * S + k] += ll.d[M + k];
    if (sn)
      for (int k = 0; k < S; ++k) grad[M + w * S + k] += ll.d[M + S + k];
  }
  total += limit_logprior(P, x, grad);
  return total;
}

// A set of R trajectories, each with its own shooting states: particle x =
// [theta, s^s of trajectory 0, .., s^s of trajectory R-1].  Each
// trajectory's log p_ms,r (Eq. 5) comes from particle_loglik_grad on a
// one-trajectory view of the problem; the parameter-limit prior is counted
// once.  Sum (Eq. traj_likelihood_sum, equally weighted: the mixture's 1/R):
//   log p = logsumexp_r(a_r) - log R + log p_lim,  a_r = log p_ms,r - log p_lim
//   d log p = sum_r w_r d a_r + d log p_lim,        w = softmax(a)
// Product (Eq. traj_likelihood_prod):  log p = sum_r a_r + log p_lim.
static double set_loglik_grad(const Problem& P, const double* x, double* grad) {
  const int S = 2 * P.n, M = P.M, W = P.W, R = P.R;
  const int Ps = (W - 1) * S, P1 = M + Ps, Pdim = M + R * Ps;
  Problem one = P;
  one.R = 1;
  std::vector<double> xr(P1), gr(P1), a(R), gprior(M, 0.0);
  std::vector<std::vector<double>> grads(R);
  const double prior = limit_logprior(P, x, gprior.data());
  for (int r = 0; r < R; ++r) {
    one.obs = P.obs + (size_t)r * P.T * P.D;
    one.s0 = P.s0 + (size_t)r * S;
    std::copy(x, x + M, xr.begin());
    std::copy(x + M + r * Ps, x + M + (r + 1) * Ps, xr.begin() + M);
    a[r] = particle_loglik_grad(one, xr.data(), grad ? gr.data() : nullptr) - prior;
    if (grad) {
      grads[r] = gr;
      for (int k = 0; k < M; ++k) grads[r][k] -= gprior[k];
    }
  }
  std::vector<double> w(R, 1.0);
  double lp = 0.0;
  if (P.combine == 0) {
    const double amax = *std::max_element(a.begin(), a.end());
    double z = 0.0;
    for (int r = 0; r < R; ++r) z += std::exp(a[r] - amax);
    lp = amax + std::log(z) - std::log((double)R);
    for (int r = 0; r < R; ++r) w[r] = std::exp(a[r] - amax) / z;
  } else {
    for (int r = 0; r < R; ++r) lp += a[r];
  }
  if (grad) {
    std::fill(grad, grad + Pdim, 0.0);
    for (int k = 0; k < M; ++k) {
      grad[k] = gprior[k];
      for (int r = 0; r < R; ++r) grad[k] += w[r] * grads[r][k];
    }
    for (int r = 0; r < R; ++r)
      for (int k = 0; k < Ps; ++k) grad[M + r * Ps + k] = w[r] * grads[r][M + k];
  }
  return lp + prior;
}

// ---------------------------------------------------------------------------
// Constrained SVGD (Sec. IV-E, Eq. mdmm-loss, Algorithm 1): the likelihood is
// the observation term only; the defect and limit terms become equality
// constraints handled by MDMM with per-particle multipliers.
//   g_def,w = ||s^s_w - s_end(w-1)||^2 / sigma_def^2      (w = 1..W-1)
//   g_lim,k = clamp(u_k, 0, 1) - u_k,  u = (theta - lo) / (hi - lo)
//   Psi     = sum_w (lam_def,w g_def,w + c/2 g_def,w^2)
//           + sum_k (lam_lim,k g_lim,k + c/2 g_lim,k^2)
// with the multipliers held fixed, so that the MDMM flow is
//   theta' = phi(theta) - dPsi/dtheta,  s' = d(log p_obs - Psi)/ds,
//   lam'   = g.
// ---------------------------------------------------------------------------
// The window's observation log-likelihood and, for w < W-1, the defect
// constraint value g_def,w+1 (the two parts of window_loglik, kept apart).
template <class T>
static void window_obs_and_defect(const Problem& P, const T* m, const T* l, const T* b, const T* s_start,
                                  const T* s_next, int w, T* obs_ll, T* gdef) {
  const int n = P.n, S = 2 * n;
  Chain<T> ch{n, m, l, b, P.g};
  std::vector<T> s(s_start, s_start + S), sn(S);
  const int t0 = window_start(P, w), t1 = window_start(P, w + 1);
  const double so2 = P.sigma_obs * P.sigma_obs;
  const double obs_const = -0.5 * P.D * std::log(2.0 * M_PI * so2);
  T ll(0.0);
  for (int t = t0 + 1; t <= t1; ++t) {
    step(ch, P.dt, s.data(), sn.data());
    s.swap(sn);
    T acc(0.0);
    for (int k = 0; k < P.D; ++k) {
      T r = T(P.obs[(size_t)(t - 1) * P.D + k]) - s[P.obs_index[k]];
      acc += r * r;
    }
    ll += acc * T(-0.5 / so2) + T(obs_const);
  }
  *obs_ll = ll;
  T g(0.0);
  if (w < P.W - 1) {
    for (int k = 0; k < S; ++k) {
      T d = s_next[k] - s[k];
      g += d * d;
    }
    g = g * T(1.0 / (P.sigma_def * P.sigma_def));
  }
  *gdef = g;
}

// One particle x = [theta (M), s^s_1..s^s_{W-1} (S each), lam_def (W-1),
// lam_lim (M)]: returns log p_obs and writes out[Pc + M]:
//   [0, M)                  d log p_obs / d theta
//   [M, M + (W-1) S)        d (log p_obs - Psi) / d s^s
//   [.., + (W-1))           g_def,w        (the lam_def flow)
//   [.., + M)               g_lim,k        (the lam_lim flow)
//   [Pc, Pc + M)            - dPsi / d theta
static double particle_csvgd(const Problem& P, double c, const double* x, double* out) {
  const int n = P.n, S = 2 * n, M = P.M, W = P.W;
  const int Pms = M + (W - 1) * S, Pc = Pms + (W - 1) + M;
  std::fill(out, out + Pc + M, 0.0);
  const double* lam_def = x + Pms;
  const double* lam_lim = x + Pms + (W - 1);
  double total = 0.0;
  for (int w = 0; w < W; ++w) {
    const double* ss = (w == 0) ? P.s0 : x + M + (w - 1) * S;
    const double* sn = (w < W - 1) ? x + M + w * S : nullptr;
    g_nd = M + 2 * S;
    std::vector<Dual> th(M), s_start(S), s_next(S);
    for (int k = 0; k < M; ++k) { th[k] = Dual(x[k]); th[k].d[k] = 1.0; }
    for (int k = 0; k < S; ++k) {
      s_start[k] = Dual(ss[k]);
      if (w > 0) s_start[k].d[M + k] = 1.0;
      if (sn) { s_next[k] = Dual(sn[k]); s_next[k].d[M + S + k] = 1.0; }
    }
    std::vector<Dual> m, l, b;
    physical_params<Dual>(P, th.data(), m, l, b);
    Dual ll, g;
    window_obs_and_defect<Dual>(P, m.data(), l.data(), b.data(), s_start.data(), sn ? s_next.data() : nullptr, w,
                                &ll, &g);
    total += ll.v;
    for (int k = 0; k < M; ++k) out[k] += ll.d[k];
    if (w > 0)
      for (int k = 0; k < S; ++k) out[M + (w - 1) * S + k] += ll.d[M + k];
    if (sn) {
      // constraint g_def,w+1 with multiplier lam_def[w]: -dPsi = -(lam + c g) dg
      const double kappa = lam_def[w] + c * g.v;
      out[Pms + w] = g.v;
      for (int k = 0; k < M; ++k) out[Pc + k] -= kappa * g.d[k];
      if (w > 0)
        for (int k = 0; k < S; ++k) out[M + (w - 1) * S + k] -= kappa * g.d[M + k];
      for (int k = 0; k < S; ++k) out[M + w * S + k] -= kappa * g.d[M + S + k];
    }
  }
  for (int k = 0; k < M; ++k) {
    const double wd = P.hi[k] - P.lo[k];
    const double u = (x[k] - P.lo[k]) / wd;
    const double gl = std::min(1.0, std::max(0.0, u)) - u;
    const double dg_du = (u < 0.0 || u > 1.0) ? -1.0 : 0.0;  // d clamp / du is 0 outside the box
    out[Pms + (W - 1) + k] = gl;
    out[Pc + k] -= (lam_lim[k] + c * gl) * dg_du / wd;
  }
  return total;
}

// ---------------------------------------------------------------------------
// SVGD (Eq. 1) with RBF kernel on unit-box coordinates and Adam ascent.
// ---------------------------------------------------------------------------
// Lower median of the N(N-1)/2 squared distances d_ij (i<j).
static double median_sqdist(int N, int M, const double* u /*[N][M]*/) {
  if (N < 2) return 0.0;
  std::vector<double> d;
  d.reserve((size_t)N * (N - 1) / 2);
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j) {
      double s = 0.0;
      for (int k = 0; k < M; ++k) {
        const double e = u[(size_t)i * M + k] - u[(size_t)j * M + k];
        s += e * e;
      }
      d.push_back(s);
    }
  const size_t r = (d.size() - 1) / 2;
  std::nth_element(d.begin(), d.begin() + r, d.end());
  return d[r];
}

static double bandwidth_from_median(int N, double med) {
  if (N < 2 || !(med > 0.0)) return 1.0;
  return med / std::log((double)N);
}

// phi_i = 1/N sum_j [ k(u_j,u_i) g_j + grad_{u_j} k(u_j,u_i) ],
// k(a,b) = exp(-||a-b||^2 / bw), grad_{u_j} k(u_j,u_i) = (2/bw)(u_i-u_j) k.
// phi of particle i (Eq. 1): (1/N) sum_j k_ij [g_j + (2/bw)(u_i - u_j)].
static void svgd_phi_row(int i, int N, int M, const double* u, const double* g, double bw, double* phi_i) {
  for (int k = 0; k < M; ++k) phi_i[k] = 0.0;
  for (int j = 0; j < N; ++j) {
    double d = 0.0;
    for (int k = 0; k < M; ++k) {
      const double e = u[(size_t)i * M + k] - u[(size_t)j * M + k];
      d += e * e;
    }
    const double kij = std::exp(-d / bw);
    for (int k = 0; k < M; ++k)
      phi_i[k] += kij * g[(size_t)j * M + k] + (2.0 / bw) * (u[(size_t)i * M + k] - u[(size_t)j * M + k]) * kij;
  }
  for (int k = 0; k < M; ++k) phi_i[k] /= N;
}

static void svgd_phi(int N, int M, const double* u, const double* g, double bw, double* phi) {
  for (int i = 0; i < N; ++i) svgd_phi_row(i, N, M, u, g, bw, phi + (size_t)i * M);
}

// Particles that sit out an SVGD step: any unit-box coordinate or gradient
// component not finite.  They take no part in the median's pairs or in the
// other particles' sums; the bandwidth and the 1/N of Eq. 1 count the live
// particles only, and a particle that sits out gets the direction NaN.
static int live_mask(int N, int M, const double* u, const double* g, std::vector<char>& live) {
  live.assign(N, 1);
  int n = 0;
  for (int i = 0; i < N; ++i) {
    for (int k = 0; k < M; ++k)
      if (!std::isfinite(u[(size_t)i * M + k]) || !std::isfinite(g[(size_t)i * M + k])) live[i] = 0;
    n += live[i];
  }
  return n;
}

// Median (as median_sqdist) and phi (as svgd_phi) over the live particles.
static double live_step_phi(int N, int M, const double* u, const double* g, double* phi, double* bw_out) {
  std::vector<char> live;
  const int nl = live_mask(N, M, u, g, live);
  std::vector<double> ul, gl;
  std::vector<int> idx;
  for (int i = 0; i < N; ++i)
    if (live[i]) {
      idx.push_back(i);
      for (int k = 0; k < M; ++k) { ul.push_back(u[(size_t)i * M + k]); gl.push_back(g[(size_t)i * M + k]); }
    }
  const double bw = bandwidth_from_median(nl, median_sqdist(nl, M, ul.data()));
  std::vector<double> pl((size_t)nl * M);
  if (nl > 0) svgd_phi(nl, M, ul.data(), gl.data(), bw, pl.data());
  for (size_t t = 0; t < (size_t)N * M; ++t) phi[t] = std::numeric_limits<double>::quiet_NaN();
  for (int a = 0; a < nl; ++a)
    for (int k = 0; k < M; ++k) phi[(size_t)idx[a] * M + k] = pl[(size_t)a * M + k];
  *bw_out = bw;
  return bw;
}

// Adam ascent on x with direction g (Kingma & Ba): bias-corrected moments.
static void adam_ascent(double& x, double& m, double& v, double g, int t, double lr, double b1, double b2, double eps) {
  m = b1 * m + (1.0 - b1) * g;
  v = b2 * v + (1.0 - b2) * g * g;
  const double mh = m / (1.0 - std::pow(b1, t));
  const double vh = v / (1.0 - std::pow(b2, t));
  x += lr * mh / (std::sqrt(vh) + eps);
}


// ---------------------------------------------------------------------------
// Arm shaking a box (Sec. V-C, Panda arm experiment, synthetic analogue).
// A serial arm of revolute joints with prescribed motion carries, at its
// end, a box hanging on two passive revolute joints (a U-joint: axis x, then
// axis y, both at the same point).  The box is a solid cube plus two point
// weights whose (x, y) positions are theta.  Only the two box joints are
// simulated; the arm is a moving base whose velocity and acceleration follow
// from its prescribed joint trajectories.
// 6-D spatial algebra (Featherstone): motion (w; v), force (n; f).
// ---------------------------------------------------------------------------
template <class T> struct V6 { T a[6]; };
template <class T> struct M6 { T a[6][6]; };
template <class T> struct R3 { T a[3][3]; };

template <class T> static V6<T> v6zero() { V6<T> r; for (int i = 0; i < 6; ++i) r.a[i] = T(0.0); return r; }
template <class T> static M6<T> m6zero() { M6<T> r; for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) r.a[i][j] = T(0.0); return r; }

template <class T> static V6<T> mul6(const M6<T>& m, const V6<T>& v) {
  V6<T> r;
  for (int i = 0; i < 6; ++i) { T s(0.0); for (int j = 0; j < 6; ++j) s += m.a[i][j] * v.a[j]; r.a[i] = s; }
  return r;
}
template <class T> static V6<T> mul6T(const M6<T>& m, const V6<T>& v) {
  V6<T> r;
  for (int i = 0; i < 6; ++i) { T s(0.0); for (int j = 0; j < 6; ++j) s += m.a[j][i] * v.a[j]; r.a[i] = s; }
  return r;
}
template <class T> static M6<T> mm6(const M6<T>& x, const M6<T>& y) {
  M6<T> r;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) { T s(0.0); for (int k = 0; k < 6; ++k) s += x.a[i][k] * y.a[k][j]; r.a[i][j] = s; }
  return r;
}
template <class T> static M6<T> tr6(const M6<T>& x) { M6<T> r; for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) r.a[i][j] = x.a[j][i]; return r; }
template <class T> static V6<T> add6(const V6<T>& x, const V6<T>& y) { V6<T> r; for (int i = 0; i < 6; ++i) r.a[i] = x.a[i] + y.a[i]; return r; }
template <class T> static M6<T> madd6(const M6<T>& x, const M6<T>& y) { M6<T> r; for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) r.a[i][j] = x.a[i][j] + y.a[i][j]; return r; }

// coordinate rotation about a principal axis (Featherstone's rx, ry, rz)
template <class T> static R3<T> rot_axis(int axis, const T& q) {
  T c = cos(q), s = sin(q);
  R3<T> E;
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) E.a[i][j] = T(i == j ? 1.0 : 0.0);
  const int i1 = (axis + 1) % 3, i2 = (axis + 2) % 3;
  E.a[i1][i1] = c; E.a[i1][i2] = s;
  E.a[i2][i1] = -s; E.a[i2][i2] = c;
  return E;
}
// Plucker transform for a frame rotated by E (coordinate transform) and
// translated by r (in the parent frame): X = [E 0; -E rx E].
template <class T> static M6<T> plux(const R3<T>& E, const T* r) {
  M6<T> X = m6zero<T>();
  T rx[3][3] = {{T(0.0), -r[2], r[1]}, {r[2], T(0.0), -r[0]}, {-r[1], r[0], T(0.0)}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      X.a[i][j] = E.a[i][j];
      X.a[3 + i][3 + j] = E.a[i][j];
      T s(0.0);
      for (int k = 0; k < 3; ++k) s += E.a[i][k] * rx[k][j];
      X.a[3 + i][j] = -s;
    }
  return X;
}
template <class T> static V6<T> crm6(const V6<T>& v, const V6<T>& m) {  // v x m
  V6<T> r;
  const T *w = v.a, *vo = v.a + 3, *mw = m.a, *mv = m.a + 3;
  r.a[0] = w[1] * mw[2] - w[2] * mw[1];
  r.a[1] = w[2] * mw[0] - w[0] * mw[2];
  r.a[2] = w[0] * mw[1] - w[1] * mw[0];
  r.a[3] = w[1] * mv[2] - w[2] * mv[1] + vo[1] * mw[2] - vo[2] * mw[1];
  r.a[4] = w[2] * mv[0] - w[0] * mv[2] + vo[2] * mw[0] - vo[0] * mw[2];
  r.a[5] = w[0] * mv[1] - w[1] * mv[0] + vo[0] * mw[1] - vo[1] * mw[0];
  return r;
}
template <class T> static V6<T> crf6(const V6<T>& v, const V6<T>& f) {  // v x* f
  V6<T> r;
  const T *w = v.a, *vo = v.a + 3, *n = f.a, *fo = f.a + 3;
  r.a[0] = w[1] * n[2] - w[2] * n[1] + vo[1] * fo[2] - vo[2] * fo[1];
  r.a[1] = w[2] * n[0] - w[0] * n[2] + vo[2] * fo[0] - vo[0] * fo[2];
  r.a[2] = w[0] * n[1] - w[1] * n[0] + vo[0] * fo[1] - vo[1] * fo[0];
  r.a[3] = w[1] * fo[2] - w[2] * fo[1];
  r.a[4] = w[2] * fo[0] - w[0] * fo[2];
  r.a[5] = w[0] * fo[1] - w[1] * fo[0];
  return r;
}
// rigid-body inertia of mass m with COM c and rotational inertia Ic (about the COM)
template <class T> static M6<T> mcI(const T& m, const T* c, const T (&Ic)[3][3]) {
  M6<T> I = m6zero<T>();
  T cx[3][3] = {{T(0.0), -c[2], c[1]}, {c[2], T(0.0), -c[0]}, {-c[1], c[0], T(0.0)}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T s(0.0);
      for (int k = 0; k < 3; ++k) s += cx[i][k] * cx[j][k];  // cx cx^T
      I.a[i][j] = Ic[i][j] + m * s;
      I.a[i][3 + j] = m * cx[i][j];
      I.a[3 + i][j] = m * cx[j][i];
      I.a[3 + i][3 + j] = T(i == j ? 1.0 : 0.0) * m;
    }
  return I;
}

struct ArmBox {
  int n_arm;              // prescribed arm joints; axes alternate z, y, z, ...
  const double* arm_len;  // [n_arm] offset to the next joint along the local z axis
  const double* amp;      // [n_arm][3] sinusoid amplitudes [rad]
  const double* freq;     // [n_arm][3] [Hz]
  const double* phase;    // [n_arm][3] [rad]
  double box_mass, box_side, box_com_depth;
  double weight_mass0, weight_mass1, weight_depth;
  double g, damping;
};

// Prescribed arm joint angle and its first two time derivatives.
static void arm_joint(const ArmBox& A, int j, double t, double* q, double* qd, double* qdd) {
  *q = *qd = *qdd = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double a = A.amp[3 * j + k], w = 2.0 * M_PI * A.freq[3 * j + k], ph = A.phase[3 * j + k];
    *q += a * std::sin(w * t + ph);
    *qd += a * w * std::cos(w * t + ph);
    *qdd += -a * w * w * std::sin(w * t + ph);
  }
}

// Spatial velocity and acceleration (acceleration offset by -gravity, as
// the articulated-body algorithm's base acceleration) of the box pivot frame
// at time t, in pivot coordinates, by the recursive kinematics of the arm.
static void arm_pivot_motion(const ArmBox& A, double t, V6<double>* v_out, V6<double>* a_out) {
  V6<double> v = v6zero<double>(), a = v6zero<double>();
  a.a[5] = A.g;  // -gravity (gravity along -z of the world)
  double zero3[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < A.n_arm; ++j) {
    double q, qd, qdd;
    arm_joint(A, j, t, &q, &qd, &qdd);
    const int axis = (j % 2 == 0) ? 2 : 1;  // z, y, z, y, ...
    double r[3] = {0.0, 0.0, j == 0 ? 0.0 : A.arm_len[j - 1]};
    M6<double> Xup = mm6(plux<double>(rot_axis<double>(axis, q), zero3), plux<double>(rot_axis<double>(0, 0.0), r));
    V6<double> S = v6zero<double>();
    S.a[axis] = 1.0;
    V6<double> vJ = S;
    for (int i = 0; i < 6; ++i) vJ.a[i] *= qd;
    v = add6(mul6(Xup, v), vJ);
    V6<double> aJ = S;
    for (int i = 0; i < 6; ++i) aJ.a[i] *= qdd;
    a = add6(add6(mul6(Xup, a), aJ), crm6(v, vJ));
  }
  // pivot: the tip of the last link
  double r[3] = {0.0, 0.0, A.arm_len[A.n_arm - 1]};
  M6<double> X = plux<double>(rot_axis<double>(0, 0.0), r);
  *v_out = mul6(X, v);
  *a_out = mul6(X, a);
}

// Spatial inertia of the box (cube + two point weights at (x_k, y_k, -depth)).
template <class T>
static M6<T> box_inertia(const ArmBox& A, const T* th) {
  const double side = A.box_side, m = A.box_mass;
  T Ic[3][3];
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) Ic[i][j] = T(i == j ? m * side * side / 6.0 : 0.0);
  T c[3] = {T(0.0), T(0.0), T(-A.box_com_depth)};
  M6<T> I = mcI<T>(T(m), c, Ic);
  T Z[3][3];
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) Z[i][j] = T(0.0);
  T p0[3] = {th[0], th[1], T(-A.weight_depth)};
  T p1[3] = {th[2], th[3], T(-A.weight_depth)};
  I = madd6(I, mcI<T>(T(A.weight_mass0), p0, Z));
  I = madd6(I, mcI<T>(T(A.weight_mass1), p1, Z));
  return I;
}

// ABA for the two box joints (body 1: massless, joint about x; body 2: the
// box, joint about y, same origin) on a base with spatial velocity v0 and
// acceleration a0 (a0 already offset by -gravity).
template <class T>
static void box_aba(const ArmBox& A, const M6<T>& Ibox, const T* q, const T* qd, const T* tau, const V6<double>& v0,
                    const V6<double>& a0, T* qdd) {
  T zero3[3] = {T(0.0), T(0.0), T(0.0)};
  M6<T> Xup[2];
  Xup[0] = plux<T>(rot_axis<T>(0, q[0]), zero3);
  Xup[1] = plux<T>(rot_axis<T>(1, q[1]), zero3);
  V6<T> S[2];
  S[0] = v6zero<T>(); S[0].a[0] = T(1.0);
  S[1] = v6zero<T>(); S[1].a[1] = T(1.0);
  V6<T> vb, ab;
  for (int i = 0; i < 6; ++i) { vb.a[i] = T(v0.a[i]); ab.a[i] = T(a0.a[i]); }
  V6<T> v[2], c[2], pA[2], U[2], a[2];
  M6<T> IA[2];
  T d[2], u[2];
  for (int i = 0; i < 2; ++i) {
    V6<T> vJ = S[i];
    for (int k = 0; k < 6; ++k) vJ.a[k] = vJ.a[k] * qd[i];
    v[i] = add6(mul6(Xup[i], i == 0 ? vb : v[i - 1]), vJ);
    c[i] = crm6(v[i], vJ);
    IA[i] = (i == 1) ? Ibox : m6zero<T>();
    pA[i] = crf6(v[i], mul6(IA[i], v[i]));
  }
  for (int i = 1; i >= 0; --i) {
    U[i] = mul6(IA[i], S[i]);
    d[i] = S[i].a[0] * U[i].a[0] + S[i].a[1] * U[i].a[1];  // S has one non-zero entry
    T sp(0.0);
    for (int k = 0; k < 6; ++k) sp += S[i].a[k] * pA[i].a[k];
    u[i] = tau[i] - sp;
    if (i > 0) {
      M6<T> Ia;
      for (int r = 0; r < 6; ++r) for (int s2 = 0; s2 < 6; ++s2) Ia.a[r][s2] = IA[i].a[r][s2] - U[i].a[r] * U[i].a[s2] / d[i];
      V6<T> pa = mul6(Ia, c[i]);
      for (int r = 0; r < 6; ++r) pa.a[r] = pA[i].a[r] + pa.a[r] + U[i].a[r] * u[i] / d[i];
      IA[i - 1] = madd6(IA[i - 1], mm6(tr6(Xup[i]), mm6(Ia, Xup[i])));
      pA[i - 1] = add6(pA[i - 1], mul6T(Xup[i], pa));
    }
  }
  for (int i = 0; i < 2; ++i) {
    a[i] = add6(mul6(Xup[i], i == 0 ? ab : a[i - 1]), c[i]);
    T ua(0.0);
    for (int k = 0; k < 6; ++k) ua += U[i].a[k] * a[i].a[k];
    qdd[i] = (u[i] - ua) / d[i];
    for (int k = 0; k < 6; ++k) a[i].a[k] = a[i].a[k] + S[i].a[k] * qdd[i];
  }
}

// One semi-implicit Euler step of the box at time t (state [q1, q2, qd1, qd2]).
template <class T>
static void box_step(const ArmBox& A, const M6<T>& Ibox, double t, double dt, const T* s, T* sn) {
  V6<double> v0, a0;
  arm_pivot_motion(A, t, &v0, &a0);
  T tau[2] = {-(T(A.damping) * s[2]), -(T(A.damping) * s[3])};
  T qdd[2];
  box_aba<T>(A, Ibox, s, s + 2, tau, v0, a0, qdd);
  for (int i = 0; i < 2; ++i) {
    T v = s[2 + i] + qdd[i] * T(dt);
    sn[2 + i] = v;
    sn[i] = s[i] + v * T(dt);
  }
}

struct ArmBoxProblem {
  ArmBox ab;
  double dt;
  int T, W, D;
  const int* obs_index;   // [D] into the box state [q1, q2, qd1, qd2]
  const double* obs;      // [T][D], row t-1 holds x_t
  double sigma_obs, sigma_def;
  const double* s0;       // [4]
  const double* lo;       // [4]
  const double* hi;       // [4]
  double c_lim;
};

template <class T>
static T armbox_window(const ArmBoxProblem& P, const T* th, const T* s_start, const T* s_next, int w) {
  const M6<T> Ibox = box_inertia<T>(P.ab, th);
  std::vector<T> s(s_start, s_start + 4), sn(4);
  const int t0 = (int)(((long long)w * P.T) / P.W), t1 = (int)(((long long)(w + 1) * P.T) / P.W);
  const double so2 = P.sigma_obs * P.sigma_obs;
  const double obs_const = -0.5 * P.D * std::log(2.0 * M_PI * so2);
  T ll(0.0);
  for (int t = t0 + 1; t <= t1; ++t) {
    box_step<T>(P.ab, Ibox, (t - 1) * P.dt, P.dt, s.data(), sn.data());
    s.swap(sn);
    T acc(0.0);
    for (int k = 0; k < P.D; ++k) {
      T r = T(P.obs[(size_t)(t - 1) * P.D + k]) - s[P.obs_index[k]];
      acc += r * r;
    }
    ll += acc * T(-0.5 / so2) + T(obs_const);
  }
  if (w < P.W - 1) {
    const double sd2 = P.sigma_def * P.sigma_def;
    T acc(0.0);
    for (int k = 0; k < 4; ++k) {
      T d = s_next[k] - s[k];
      acc += d * d;
    }
    ll += acc * T(-0.5 / sd2) + T(-0.5 * 4 * std::log(2.0 * M_PI * sd2));
  }
  return ll;
}

static double armbox_particle(const ArmBoxProblem& P, const double* x, double* grad) {
  const int M = 4, S = 4, W = P.W, Pdim = M + (W - 1) * S;
  if (grad) std::fill(grad, grad + Pdim, 0.0);
  double total = 0.0;
  for (int w = 0; w < W; ++w) {
    const double* ss = (w == 0) ? P.s0 : x + M + (w - 1) * S;
    const double* sn = (w < W - 1) ? x + M + w * S : nullptr;
    if (!grad) {
      total += armbox_window<double>(P, x, ss, sn, w);
      continue;
    }
    g_nd = M + 2 * S;
    std::vector<Dual> th(M), a(S), b(S);
    for (int k = 0; k < M; ++k) { th[k] = Dual(x[k]); th[k].d[k] = 1.0; }
    for (int k = 0; k < S; ++k) {
      a[k] = Dual(ss[k]);
      if (w > 0) a[k].d[M + k] = 1.0;
      if (sn) { b[k] = Dual(sn[k]); b[k].d[M + S + k] = 1.0; }
    }
    Dual ll = armbox_window<Dual>(P, th.data(), a.data(), sn ? b.data() : nullptr, w);
    total += ll.v;
    for (int k = 0; k < M; ++k) grad[k] += ll.d[k];
    if (w > 0) for (int k = 0; k < S; ++k) grad[M + (w - 1) * S + k] += ll.d[M + k];
    if (sn) for (int k = 0; k < S; ++k) grad[M + w * S + k] += ll.d[M + S + k];
  }
  // limit prior, as for the chain problems
  for (int k = 0; k < M; ++k) {
    const double wd = P.hi[k] - P.lo[k];
    const double u = (x[k] - P.lo[k]) / wd;
    const double cu = std::min(1.0, std::max(0.0, u));
    total += -std::log(wd) - 0.5 * P.c_lim * (cu - u) * (cu - u);
    if (grad) grad[k] += P.c_lim * (cu - u) / wd;
  }
  return total;
}

// ---------------------------------------------------------------------------
// Rigid double pendulum with general inertia and centre of mass (the
// 11-parameter physical double pendulum of Sec. V's real-world experiment,
// App. Table params-ibm-pendulum), by the 6-D articulated-body algorithm.
// Two rigid links on revolute joints about their frames' z axes; joint 1 at
// the world origin, joint 2 at (0, -l, 0) in link 1's frame; link k has
// mass m_k, centre of mass c_k (link frame) and rotational inertia Ic_k (3x3,
// about the COM); viscous joint friction tau_k = -b_k qd_k; gravity along
// -y.  State [q1, q2, qd1, qd2]; q = 0 with c_k along -y hangs at rest.
// The 11 estimated parameters, in the table's order:
//   [m1, I1, c1x, c1y, b1, l, m2, I2, c2x, c2y, b2]
// with c_k = (ckx, cky, 0) and Ic_k = I_k times the identity.
// ---------------------------------------------------------------------------
struct Rigid2 {
  double p[11];  // nominal values of all parameters
  double g;
};

template <class T>
static void rigid2_aba(const T* m, const T (*c)[3], const T (*Ic)[3][3], const T* b, const T& l, double g, const T* s,
                       T* qdd) {
  T zero3[3] = {T(0.0), T(0.0), T(0.0)};
  T r2[3] = {T(0.0), -l, T(0.0)};
  R3<T> Id;
  for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) Id.a[i][j] = T(i == j ? 1.0 : 0.0);
  M6<T> Xup[2];
  Xup[0] = plux<T>(rot_axis<T>(2, s[0]), zero3);
  Xup[1] = mm6(plux<T>(rot_axis<T>(2, s[1]), zero3), plux<T>(Id, r2));
  V6<T> S = v6zero<T>();
  S.a[2] = T(1.0);
  V6<T> a0 = v6zero<T>();
  a0.a[4] = T(g);  // base acceleration = -gravity (gravity along -y)
  V6<T> v[2], cc[2], pA[2], U[2], a[2];
  M6<T> IA[2];
  T d[2], u[2];
  for (int i = 0; i < 2; ++i) {
    V6<T> vJ = S;
    for (int k = 0; k < 6; ++k) vJ.a[k] = vJ.a[k] * s[2 + i];
    v[i] = (i == 0) ? vJ : add6(mul6(Xup[i], v[i - 1]), vJ);
    cc[i] = crm6(v[i], vJ);
    T Ick[3][3];
    for (int r = 0; r < 3; ++r) for (int q = 0; q < 3; ++q) Ick[r][q] = Ic[i][r][q];
    IA[i] = mcI<T>(m[i], c[i], Ick);
    pA[i] = crf6(v[i], mul6(IA[i], v[i]));
  }
  for (int i = 1; i >= 0; --i) {
    U[i] = mul6(IA[i], S);
    d[i] = U[i].a[2];
    u[i] = -(b[i] * s[2 + i]) - pA[i].a[2];
    if (i > 0) {
      M6<T> Ia;
      for (int r = 0; r < 6; ++r) for (int q = 0; q < 6; ++q) Ia.a[r][q] = IA[i].a[r][q] - U[i].a[r] * U[i].a[q] / d[i];
      V6<T> pa = mul6(Ia, cc[i]);
      for (int r = 0; r < 6; ++r) pa.a[r] = pA[i].a[r] + pa.a[r] + U[i].a[r] * u[i] / d[i];
      IA[i - 1] = madd6(IA[i - 1], mm6(tr6(Xup[i]), mm6(Ia, Xup[i])));
      pA[i - 1] = add6(pA[i - 1], mul6T(Xup[i], pa));
    }
  }
  for (int i = 0; i < 2; ++i) {
    a[i] = add6(mul6(Xup[i], i == 0 ? a0 : a[i - 1]), cc[i]);
    T ua(0.0);
    for (int k = 0; k < 6; ++k) ua += U[i].a[k] * a[i].a[k];
    qdd[i] = (u[i] - ua) / d[i];
    for (int k = 0; k < 6; ++k) a[i].a[k] = a[i].a[k] + S.a[k] * qdd[i];
  }
}

// The 11-parameter form: c_k = (ckx, cky, 0), Ic_k = I_k identity.
template <class T>
static void rigid2_qdd(const T* p, double g, const T* s, T* qdd) {
  T m[2] = {p[0], p[6]}, b[2] = {p[4], p[10]};
  T c[2][3] = {{p[2], p[3], T(0.0)}, {p[8], p[9], T(0.0)}};
  T Ic[2][3][3];
  for (int k = 0; k < 2; ++k)
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) Ic[k][i][j] = (i == j) ? p[k == 0 ? 1 : 7] : T(0.0);
  rigid2_aba<T>(m, c, Ic, b, p[5], g, s, qdd);
}

template <class T>
static void rigid2_step(const T* p, double g, double dt, const T* s, T* sn) {
  T qdd[2];
  rigid2_qdd<T>(p, g, s, qdd);
  for (int i = 0; i < 2; ++i) {
    T v = s[2 + i] + qdd[i] * T(dt);
    sn[2 + i] = v;
    sn[i] = s[i] + v * T(dt);
  }
}

struct Rigid2Problem {
  Rigid2 sys;
  int M;
  const int* theta_param;  // [M] indices into the 11 parameters
  double dt;
  int T, W, D;
  const int* obs_index;    // [D] into the state
  const double* obs;       // [T][D], row t-1 holds x_t
  double sigma_obs, sigma_def;
  const double* s0;        // [4]
  const double* lo;        // [M]
  const double* hi;        // [M]
  double c_lim;
};

template <class T>
static T rigid2_window(const Rigid2Problem& P, const T* th, const T* s_start, const T* s_next, int w) {
  T p[11];
  for (int k = 0; k < 11; ++k) p[k] = T(P.sys.p[k]);
  for (int k = 0; k < P.M; ++k) p[P.theta_param[k]] = th[k];
  std::vector<T> s(s_start, s_start + 4), sn(4);
  const int t0 = (int)(((long long)w * P.T) / P.W), t1 = (int)(((long long)(w + 1) * P.T) / P.W);
  const double so2 = P.sigma_obs * P.sigma_obs;
  const double obs_const = -0.5 * P.D * std::log(2.0 * M_PI * so2);
  T ll(0.0);
  for (int t = t0 + 1; t <= t1; ++t) {
    rigid2_step<T>(p, P.sys.g, P.dt, s.data(), sn.data());
    s.swap(sn);
    T acc(0.0);
    for (int k = 0; k < P.D; ++k) {
      T r = T(P.obs[(size_t)(t - 1) * P.D + k]) - s[P.obs_index[k]];
      acc += r * r;
    }
    ll += acc * T(-0.5 / so2) + T(obs_const);
  }
  if (w < P.W - 1) {
    const double sd2 = P.sigma_def * P.sigma_def;
    T acc(0.0);
    for (int k = 0; k < 4; ++k) {
      T d = s_next[k] - s[k];
      acc += d * d;
    }
    ll += acc * T(-0.5 / sd2) + T(-0.5 * 4 * std::log(2.0 * M_PI * sd2));
  }
  return ll;
}

static double rigid2_particle(const Rigid2Problem& P, const double* x, double* grad) {
  const int M = P.M, S = 4, W = P.W, Pdim = M + (W - 1) * S;
  if (grad) std::fill(grad, grad + Pdim, 0.0);
  double total = 0.0;
  for (int w = 0; w < W; ++w) {
    const double* ss = (w == 0) ? P.s0 : x + M + (w - 1) * S;
    const double* sn = (w < W - 1) ? x + M + w * S : nullptr;
    if (!grad) {
      total += rigid2_window<double>(P, x, ss, sn, w);
      continue;
    }
    g_nd = M + 2 * S;
    std::vector<Dual> th(M), a(S), b(S);
    for (int k = 0; k < M; ++k) { th[k] = Dual(x[k]); th[k].d[k] = 1.0; }
    for (int k = 0; k < S; ++k) {
      a[k] = Dual(ss[k]);
      if (w > 0) a[k].d[M + k] = 1.0;
      if (sn) { b[k] = Dual(sn[k]); b[k].d[M + S + k] = 1.0; }
    }
    Dual ll = rigid2_window<Dual>(P, th.data(), a.data(), sn ? b.data() : nullptr, w);
    total += ll.v;
    for (int k = 0; k < M; ++k) grad[k] += ll.d[k];
    if (w > 0) for (int k = 0; k < S; ++k) grad[M + (w - 1) * S + k] += ll.d[M + k];
    if (sn) for (int k = 0; k < S; ++k) grad[M + w * S + k] += ll.d[M + S + k];
  }
  for (int k = 0; k < M; ++k) {
    const double wd = P.hi[k] - P.lo[k];
    const double u = (x[k] - P.lo[k]) / wd;
    const double cu = std::min(1.0, std::max(0.0, u));
    total += -std::log(wd) - 0.5 * P.c_lim * (cu - u) * (cu - u);
    if (grad) grad[k] += P.c_lim * (cu - u) / wd;
  }
  return total;
}

}  // namespace orc

using namespace orc;

// ---------------------------------------------------------------------------
// C API (ctypes).  All arrays are row-major doubles unless stated.
// ---------------------------------------------------------------------------
extern "C" {

int orc_version() { return 1; }

// ABA: qdd for a chain with per-link mass/length/damping, torques given.
int orc_aba(int n, double g, const double* m, const double* l, const double* b,
            const double* q, const double* qd, const double* tau, double* qdd) {
  Chain<double> ch{n, m, l, b, g};
  aba(ch, q, qd, tau, qdd);
  return 0;
}

// CRBA mass matrix H [n][n] and bias C [n] (Coriolis + gravity).
int orc_crba(int n, double g, const double* m, const double* l, const double* b,
             const double* q, const double* qd, double* H, double* C) {
  Chain<double> ch{n, m, l, b, g};
  crba_bias(ch, q, qd, H, C);
  return 0;
}

// Forward dynamics by CRBA + Cholesky: qdd = H^-1 (tau - C).
int orc_fd_crba(int n, double g, const double* m, const double* l, const double* b,
                const double* q, const double* qd, const double* tau, double* qdd) {
  std::vector<double> H(n * n), C(n), rhs(n);
  Chain<double> ch{n, m, l, b, g};
  crba_bias(ch, q, qd, H.data(), C.data());
  for (int i = 0; i < n; ++i) rhs[i] = tau[i] - C[i];
  return cholesky_solve(n, H.data(), rhs.data(), qdd) ? 0 : -1;
}

// Total mechanical energy (kinetic + gravitational potential) of the chain.
double orc_energy(int n, double g, const double* m, const double* l, const double* q, const double* qd) {
  double px = 0, py = 0, vx = 0, vy = 0, phi = 0, om = 0, E = 0;
  for (int i = 0; i < n; ++i) {
    phi += q[i];
    om += qd[i];
    px += l[i] * std::sin(phi);
    py += -l[i] * std::cos(phi);
    vx += l[i] * std::cos(phi) * om;
    vy += l[i] * std::sin(phi) * om;
    E += 0.5 * m[i] * (vx * vx + vy * vy) + m[i] * g * py;
  }
  return E;
}

// f_sim: roll out T semi-implicit Euler steps from s0.  states [T+1][2n].
int orc_simulate(int n, double g, const double* m, const double* l, const double* b,
                 double dt, int T, const double* s0, double* states) {
  Chain<double> ch{n, m, l, b, g};
  const int S = 2 * n;
  std::copy(s0, s0 + S, states);
  for (int t = 0; t < T; ++t) step(ch, dt, states + (size_t)t * S, states + (size_t)(t + 1) * S);
  return 0;
}

// One step's Jacobian-free check helper: s_next = f_step(s).
int orc_step(int n, double g, const double* m, const double* l, const double* b,
             double dt, const double* s, double* s_next) {
  Chain<double> ch{n, m, l, b, g};
  step(ch, dt, s, s_next);
  return 0;
}

// Batched log p_ms + log p_lim and gradient.  particles [N][P] with
// P = M + (W-1)*2n; logp [N]; grad [N][P] or NULL.  Parallel over particles
// with `threads` OpenMP threads (<=0: library default).
int orc_loglik_grad(const Problem* prob, const double* particles, int N, double* logp, double* grad, int threads) {
  const Problem& P = *prob;
  // M theta directions plus 2S state directions must fit the dual width.
  if (P.n < 1 || P.M < 0 || P.W < 1 || P.T < P.W || P.M + 4 * P.n > MAXD || P.R < 1) return -1;
  const int Pdim = P.M + P.R * (P.W - 1) * 2 * P.n;
  if (P.R > 1) {
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < N; ++i)
      logp[i] = set_loglik_grad(P, particles + (size_t)i * Pdim, grad ? grad + (size_t)i * Pdim : nullptr);
    return 0;
  }
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int i = 0; i < N; ++i) {
    logp[i] = particle_loglik_grad(P, particles + (size_t)i * Pdim, grad ? grad + (size_t)i * Pdim : nullptr);
  }
  return 0;
}

int orc_max_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

double orc_median_sqdist(int N, int M, const double* u) { return median_sqdist(N, M, u); }
double orc_bandwidth(int N, double med) { return bandwidth_from_median(N, med); }

int orc_svgd_phi(int N, int M, const double* u, const double* g, double bw, double* phi) {
  svgd_phi(N, M, u, g, bw, phi);
  return 0;
}

// phi of the listed particles only: phi [n_rows][M] for rows[r].
int orc_svgd_phi_rows(int N, int M, const double* u, const double* g, double bw, const int* rows, int n_rows,
                      double* phi) {
  for (int r = 0; r < n_rows; ++r) {
    if (rows[r] < 0 || rows[r] >= N) return -1;
    svgd_phi_row(rows[r], N, M, u, g, bw, phi + (size_t)r * M);
  }
  return 0;
}

// The update of one Algorithm 1 iteration, given its directions: theta rows
// move by Adam ascent in unit-box coordinates on phi [N][M] (then clipped to
// the box if clamp), the shooting-state rows by Adam ascent on their own
// gradient rows grad[i][M..P-1].  adam_m, adam_v [N][P] hold theta moments in
// unit-box coordinates and shooting-state moments in state units; *t is the
// step count (incremented).  A particle that sat out has NaN in phi and
// stays NaN, like the step written out below.
int orc_svgd_update(int N, int M, int P, const double* lo, const double* hi, double* particles,
                    const double* phi, const double* grad, double* adam_m, double* adam_v, int* t, double lr,
                    double b1, double b2, double eps, int clamp) {
  *t += 1;
  for (int i = 0; i < N; ++i) {
    for (int k = 0; k < M; ++k) {
      double x = (particles[(size_t)i * P + k] - lo[k]) / (hi[k] - lo[k]);
      adam_ascent(x, adam_m[(size_t)i * P + k], adam_v[(size_t)i * P + k], phi[(size_t)i * M + k], *t, lr, b1, b2, eps);
      if (clamp) x = std::min(1.0, std::max(0.0, x));
      particles[(size_t)i * P + k] = lo[k] + x * (hi[k] - lo[k]);
    }
    for (int k = M; k < P; ++k)
      adam_ascent(particles[(size_t)i * P + k], adam_m[(size_t)i * P + k], adam_v[(size_t)i * P + k],
                  grad[(size_t)i * P + k], *t, lr, b1, b2, eps);
  }
  return 0;
}

// One SVGD + Adam iteration on particles [N][P] (first M entries theta,
// the rest shooting states), given grad = d log p / d x [N][P]: phi of
// Eq. 1 in unit-box coordinates, then the update above.
// phi_out [N][M] (unit-box coordinates) and bw_out may be NULL.
int orc_svgd_step(int N, int M, int P, const double* lo, const double* hi,
                  double* particles, const double* grad, double* adam_m, double* adam_v, int* t,
                  double lr, double b1, double b2, double eps, int clamp,
                  double* phi_out, double* bw_out) {
  std::vector<double> u((size_t)N * M), gu((size_t)N * M), phi((size_t)N * M);
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < M; ++k) {
      const double w = hi[k] - lo[k];
      u[(size_t)i * M + k] = (particles[(size_t)i * P + k] - lo[k]) / w;
      gu[(size_t)i * M + k] = grad[(size_t)i * P + k] * w;  // chain rule through u
    }
  double bw = 1.0;
  live_step_phi(N, M, u.data(), gu.data(), phi.data(), &bw);
  orc_svgd_update(N, M, P, lo, hi, particles, phi.data(), grad, adam_m, adam_v, t, lr, b1, b2, eps, clamp);
  if (phi_out) std::copy(phi.begin(), phi.end(), phi_out);
  if (bw_out) *bw_out = bw;
  return 0;
}

// CSVGD quantities of N particles [N][Pc] (Pc = M + (W-1) S + (W-1) + M) into
// out [N][Pc + M] as particle_csvgd; logp_obs [N].
int orc_csvgd_loglik_grad(const Problem* prob, double c, const double* particles, int N, double* logp_obs,
                          double* out, int threads) {
  const Problem& P = *prob;
  if (P.n < 1 || P.M < 0 || P.W < 1 || P.T < P.W || P.M + 4 * P.n > MAXD) return -1;
  const int S = 2 * P.n, Pc = P.M + (P.W - 1) * S + (P.W - 1) + P.M;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int i = 0; i < N; ++i)
    logp_obs[i] = particle_csvgd(P, c, particles + (size_t)i * Pc, out + (size_t)i * (Pc + P.M));
  return 0;
}

// One CSVGD iteration's update (Algorithm 1) from out = the rows above:
// theta moves by Adam ascent in u coordinates on phi (Eq. 1 with the
// observation gradient) plus the constraint direction -dPsi/du, without
// clipping; the shooting states by Adam ascent on their rows; the
// multipliers by a gradient-ascent step lam += lr g.
int orc_csvgd_step(int N, int M, int Pc, int n_def, const double* lo, const double* hi, double* particles,
                   const double* out, double* adam_m, double* adam_v, int* t, double lr, double b1, double b2,
                   double eps, double* phi_out, double* bw_out) {
  const int n_shoot = Pc - M - n_def - M;
  if (n_shoot < 0) return -1;
  const int G = Pc + M;
  std::vector<double> u((size_t)N * M), gu((size_t)N * M), phi((size_t)N * M);
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < M; ++k) {
      const double w = hi[k] - lo[k];
      u[(size_t)i * M + k] = (particles[(size_t)i * Pc + k] - lo[k]) / w;
      gu[(size_t)i * M + k] = out[(size_t)i * G + k] * w;
    }
  double bw = 1.0;
  live_step_phi(N, M, u.data(), gu.data(), phi.data(), &bw);
  *t += 1;
  for (int i = 0; i < N; ++i) {
    const double* o = out + (size_t)i * G;
    double* x = particles + (size_t)i * Pc;
    for (int k = 0; k < M; ++k) {
      const double w = hi[k] - lo[k];
      double uk = u[(size_t)i * M + k];
      adam_ascent(uk, adam_m[(size_t)i * Pc + k], adam_v[(size_t)i * Pc + k], phi[(size_t)i * M + k] + o[Pc + k] * w,
                  *t, lr, b1, b2, eps);
      x[k] = lo[k] + uk * w;
    }
    for (int k = M; k < M + n_shoot; ++k)
      adam_ascent(x[k], adam_m[(size_t)i * Pc + k], adam_v[(size_t)i * Pc + k], o[k], *t, lr, b1, b2, eps);
    for (int k = M + n_shoot; k < Pc; ++k) x[k] += lr * o[k];
  }
  if (phi_out) std::copy(phi.begin(), phi.end(), phi_out);
  if (bw_out) *bw_out = bw;
  return 0;
}

// ---------------------------------------------------------------------------
// Stochastic gradient Langevin dynamics with the multiple-shooting likelihood
// (the second estimator of Sec. V-B's multiple-shooting comparison; Welling
// and Teh 2011): every particle is an independent chain on the augmented
// vector,
//   u     <- u + (eps_t / 2) g_u + sqrt(eps_t) xi      (theta in unit-box u)
//   s^s   <- s^s + (eps_t / 2) g_s + sqrt(eps_t) xi
//   eps_t = a (b + t)^(-gamma),  t = 1, 2, ...
// xi ~ N(0, 1) per (step, row, particle) from a counter-based generator:
// SplitMix64 (Steele, Lea and Flood 2014) from `seed`, outputs 2k+1 and 2k+2
// for k = (t-1) P N + r N + i, turned into one normal by Box-Muller
// (u1 in (0, 1], u2 in [0, 1): sqrt(-2 ln u1) cos(2 pi u2)).
// ---------------------------------------------------------------------------
static uint64_t splitmix64_output(uint64_t seed, uint64_t index /* 1-based */) {
  uint64_t z = seed + index * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double langevin_normal(uint64_t seed, uint64_t k) {
  const uint64_t z1 = splitmix64_output(seed, 2 * k + 1), z2 = splitmix64_output(seed, 2 * k + 2);
  const double u1 = (double)((z1 >> 11) + 1) * 0x1.0p-53;
  const double u2 = (double)(z2 >> 11) * 0x1.0p-53;
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
}

// The generator's normal for (seed, k), and its underlying SplitMix64 output.
double orc_langevin_normal(uint64_t seed, uint64_t k) { return langevin_normal(seed, k); }
uint64_t orc_splitmix64(uint64_t seed, uint64_t index) { return splitmix64_output(seed, index); }

// One SGLD step of N particles [N][P] (theta rows first, M of them) with
// gradient grad [N][P]; t is the step count, incremented first.
int orc_sgld_step(int N, int M, int P, const double* lo, const double* hi, double* particles, const double* grad,
                  int* t, double a, double b, double gamma, uint64_t seed, int clamp) {
  *t += 1;
  const double eps = a * std::pow(b + *t, -gamma);
  const double sq = std::sqrt(eps);
  for (int i = 0; i < N; ++i)
    for (int r = 0; r < P; ++r) {
      const uint64_t k = ((uint64_t)(*t - 1) * P + r) * (uint64_t)N + i;
      const double xi = langevin_normal(seed, k);
      double& x = particles[(size_t)i * P + r];
      const double g = grad[(size_t)i * P + r];
      if (r < M) {
        const double w = hi[r] - lo[r];
        double u = (x - lo[r]) / w;
        u += 0.5 * eps * g * w + sq * xi;
        if (clamp) u = std::min(1.0, std::max(0.0, u));
        x = lo[r] + u * w;
      } else {
        x += 0.5 * eps * g + sq * xi;
      }
    }
  return 0;
}

// ---- arm + box -------------------------------------------------------------
// Spatial velocity and acceleration (minus gravity) of the box pivot at t.
int orc_armbox_pivot(const ArmBox* A, double t, double* v6, double* a6) {
  V6<double> v, a;
  arm_pivot_motion(*A, t, &v, &a);
  for (int i = 0; i < 6; ++i) { v6[i] = v.a[i]; a6[i] = a.a[i]; }
  return 0;
}

// Box joint accelerations for state s = [q1, q2, qd1, qd2] at time t.
int orc_armbox_qdd(const ArmBox* A, const double* theta, double t, const double* s, double* qdd) {
  M6<double> I = box_inertia<double>(*A, theta);
  V6<double> v0, a0;
  arm_pivot_motion(*A, t, &v0, &a0);
  double tau[2] = {-A->damping * s[2], -A->damping * s[3]};
  box_aba<double>(*A, I, s, s + 2, tau, v0, a0, qdd);
  return 0;
}

// Spatial inertia of the box (6x6, row-major) for weight positions theta.
int orc_armbox_inertia(const ArmBox* A, const double* theta, double* I66) {
  M6<double> I = box_inertia<double>(*A, theta);
  for (int i = 0; i < 6; ++i) for (int j = 0; j < 6; ++j) I66[6 * i + j] = I.a[i][j];
  return 0;
}

// f_sim of the box: states [T+1][4] from s0.
int orc_armbox_simulate(const ArmBox* A, const double* theta, double dt, int T, const double* s0, double* states) {
  M6<double> I = box_inertia<double>(*A, theta);
  std::copy(s0, s0 + 4, states);
  for (int t = 0; t < T; ++t) box_step<double>(*A, I, t * dt, dt, states + (size_t)t * 4, states + (size_t)(t + 1) * 4);
  return 0;
}

int orc_armbox_loglik_grad(const ArmBoxProblem* prob, const double* particles, int N, double* logp, double* grad,
                           int threads) {
  const ArmBoxProblem& P = *prob;
  if (P.W < 1 || P.T < P.W) return -1;
  const int Pdim = 4 + (P.W - 1) * 4;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int i = 0; i < N; ++i)
    logp[i] = armbox_particle(P, particles + (size_t)i * Pdim, grad ? grad + (size_t)i * Pdim : nullptr);
  return 0;
}

// ---- rigid double pendulum --------------------------------------------------
// qdd for general COMs c [2][3] and inertias Ic [2][3][3] (row-major).
int orc_rigid2_qdd_full(const double* m, const double* c, const double* Ic, const double* b, double l, double g,
                        const double* s, double* qdd) {
  double cc[2][3], II[2][3][3];
  for (int k = 0; k < 2; ++k)
    for (int i = 0; i < 3; ++i) {
      cc[k][i] = c[3 * k + i];
      for (int j = 0; j < 3; ++j) II[k][i][j] = Ic[9 * k + 3 * i + j];
    }
  rigid2_aba<double>(m, cc, II, b, l, g, s, qdd);
  return 0;
}

// qdd of the 11-parameter form.
int orc_rigid2_qdd(const double* p11, double g, const double* s, double* qdd) {
  rigid2_qdd<double>(p11, g, s, qdd);
  return 0;
}

// f_sim: states [T+1][4] from s0.
int orc_rigid2_simulate(const double* p11, double g, double dt, int T, const double* s0, double* states) {
  std::copy(s0, s0 + 4, states);
  for (int t = 0; t < T; ++t) rigid2_step<double>(p11, g, dt, states + (size_t)t * 4, states + (size_t)(t + 1) * 4);
  return 0;
}

int orc_rigid2_loglik_grad(const Rigid2Problem* prob, const double* particles, int N, double* logp, double* grad,
                           int threads) {
  const Rigid2Problem& P = *prob;
  if (P.W < 1 || P.T < P.W || P.M < 1 || P.M > 11 || P.M + 8 > MAXD) return -1;
  for (int k = 0; k < P.M; ++k)
    if (P.theta_param[k] < 0 || P.theta_param[k] > 10) return -1;
  const int Pdim = P.M + (P.W - 1) * 4;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int i = 0; i < N; ++i)
    logp[i] = rigid2_particle(P, particles + (size_t)i * Pdim, grad ? grad + (size_t)i * Pdim : nullptr);
  return 0;
}

}  // extern "C"
