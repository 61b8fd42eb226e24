// Arm shaking a box: rollout with forward tangents, and problem creation.
//
// The box hangs on a U-joint (axis x, then y, same point) at the tip of a
// prescribed arm; only the two box joints are simulated.  With the pivot's
// angular velocity omega_E, angular acceleration alpha_E and classical
// acceleration minus gravity g_E (pivot coordinates, tabulated per step),
// the joint moment the box needs about the pivot (box coordinates) is
//   M = I alpha_2 + omega_2 x (I omega_2) + h x g_2
// (Newton-Euler about a moving point; I: inertia about the pivot, h: first
// mass moment), with omega_2, alpha_2 propagated through the two joints.
// Its components along the joint axes equal the joint torques (viscous
// damping), which is linear in the joint accelerations: a 2x2 system solved
// in closed form.  Semi-implicit Euler as for the chains (Appendix B-A).
//
// Gradient: the 2-joint system has 4 parameters and a 4-dimensional start
// state per window, so tangents of the state along these 8 directions are
// carried forward through the window with the value (forward-mode chain
// rule); no adjoint tape is needed.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "pds_internal.cuh"

namespace pds {

constexpr int kTan = 8;  // theta (4) + window start state (4)

// value + 8 tangent components
struct Tn {
  float v;
  float d[kTan];
};

__device__ __forceinline__ Tn tconst(float x) {
  Tn r;
  r.v = x;
#pragma unroll
  for (int k = 0; k < kTan; ++k) r.d[k] = 0.f;
  return r;
}
__device__ __forceinline__ Tn operator+(const Tn& a, const Tn& b) {
  Tn r;
  r.v = a.v + b.v;
#pragma unroll
  for (int k = 0; k < kTan; ++k) r.d[k] = a.d[k] + b.d[k];
  return r;
}
__device__ __forceinline__ Tn operator-(const Tn& a, const Tn& b) {
  Tn r;
  r.v = a.v - b.v;
#pragma unroll
  for (int k = 0; k < kTan; ++k) r.d[k] = a.d[k] - b.d[k];
  return r;
}
__device__ __forceinline__ Tn operator*(const Tn& a, const Tn& b) {
  Tn r;
  r.v = a.v * b.v;
#pragma unroll
  for (int k = 0; k < kTan; ++k) r.d[k] = fmaf(a.d[k], b.v, a.v * b.d[k]);
  return r;
}
__device__ __forceinline__ Tn operator*(const Tn& a, float s) {
  Tn r;
  r.v = a.v * s;
#pragma unroll
  for (int k = 0; k < kTan; ++k) r.d[k] = a.d[k] * s;
  return r;
}
__device__ __forceinline__ Tn operator+(const Tn& a, float s) {
  Tn r = a;
  r.v += s;
  return r;
}
// a * b + c
__device__ __forceinline__ Tn tfma(const Tn& a, const Tn& b, const Tn& c) {
  Tn r;
  r.v = fmaf(a.v, b.v, c.v);
#pragma unroll
  for (int k = 0; k < kTan; ++k) r.d[k] = fmaf(a.d[k], b.v, fmaf(a.v, b.d[k], c.d[k]));
  return r;
}
// a * s + c with a plain float s
__device__ __forceinline__ Tn tfmas(const Tn& a, float s, const Tn& c) {
  Tn r;
  r.v = fmaf(a.v, s, c.v);
#pragma unroll
  for (int k = 0; k < kTan; ++k) r.d[k] = fmaf(a.d[k], s, c.d[k]);
  return r;
}
__device__ __forceinline__ Tn tdiv(const Tn& a, const Tn& b) {
  Tn r;
  const float ib = 1.0f / b.v;
  r.v = a.v * ib;
#pragma unroll
  for (int k = 0; k < kTan; ++k) r.d[k] = (a.d[k] - r.v * b.d[k]) * ib;
  return r;
}
template <bool FAST>
__device__ __forceinline__ void tsincos(const Tn& x, Tn& s, Tn& c) {
  float sv, cv;
  if (FAST) __sincosf(x.v, &sv, &cv);
  else sincosf(x.v, &sv, &cv);
  s.v = sv;
  c.v = cv;
#pragma unroll
  for (int k = 0; k < kTan; ++k) { s.d[k] = cv * x.d[k]; c.d[k] = -sv * x.d[k]; }
}

// Mass properties of the box about the pivot (box coordinates): first
// moment h and the 6 entries of the symmetric inertia, with tangents along
// the theta directions 0..3.
struct BoxMass {
  Tn h[3];
  Tn Ixx, Iyy, Izz, Ixy, Ixz, Iyz;
};

__device__ __forceinline__ BoxMass box_mass(const ArmBoxParams& ab, const float (&th)[4]) {
  BoxMass bm;
  const float mc = ab.box_mass, zc = -ab.box_com_depth, zw = -ab.w_depth;
  const float ic = mc * ab.box_side * ab.box_side / 6.0f;
  Tn x0 = tconst(th[0]), y0 = tconst(th[1]), x1 = tconst(th[2]), y1 = tconst(th[3]);
  x0.d[0] = 1.f; y0.d[1] = 1.f; x1.d[2] = 1.f; y1.d[3] = 1.f;
  const float m0 = ab.w_mass0, m1 = ab.w_mass1;
  bm.h[0] = x0 * m0 + x1 * m1;
  bm.h[1] = y0 * m0 + y1 * m1;
  bm.h[2] = tconst(mc * zc + (m0 + m1) * zw);
  // I = Ic + sum m (|c|^2 1 - c c^T)
  const Tn xx = x0 * x0 * m0 + x1 * x1 * m1;
  const Tn yy = y0 * y0 * m0 + y1 * y1 * m1;
  const Tn xy = x0 * y0 * m0 + x1 * y1 * m1;
  const float zz = mc * zc * zc + (m0 + m1) * zw * zw;
  bm.Ixx = yy + (ic + zz);
  bm.Iyy = xx + (ic + zz);
  bm.Izz = xx + yy + ic;
  bm.Ixy = xy * -1.f;
  bm.Ixz = (x0 * m0 + x1 * m1) * (-zw);
  bm.Iyz = (y0 * m0 + y1 * m1) * (-zw);
  // the cube's own COM offset is along z only: adds to Ixx, Iyy (done) and nothing off-diagonal
  return bm;
}

__device__ __forceinline__ void Imul(const BoxMass& b, const Tn (&x)[3], Tn (&y)[3]) {
  y[0] = tfma(b.Ixx, x[0], tfma(b.Ixy, x[1], b.Ixz * x[2]));
  y[1] = tfma(b.Ixy, x[0], tfma(b.Iyy, x[1], b.Iyz * x[2]));
  y[2] = tfma(b.Ixz, x[0], tfma(b.Iyz, x[1], b.Izz * x[2]));
}

// One semi-implicit Euler step of the box with tangents.
template <bool FAST>
__device__ __forceinline__ void box_step(const ArmBoxParams& ab, const BoxMass& bm, const float* __restrict__ base,
                                         float dt, Tn (&s)[4]) {
  const float wE0 = __ldg(base + 0), wE1 = __ldg(base + 1), wE2 = __ldg(base + 2);
  const float aE0 = __ldg(base + 3), aE1 = __ldg(base + 4), aE2 = __ldg(base + 5);
  const float gE0 = __ldg(base + 6), gE1 = __ldg(base + 7), gE2 = __ldg(base + 8);
  Tn s1, c1, s2, c2;
  tsincos<FAST>(s[0], s1, c1);
  tsincos<FAST>(s[1], s2, c2);
  const Tn v1 = s[2], v2 = s[3];
  // frame 1 (after the x joint): R1^T x = (x0, c1 x1 + s1 x2, -s1 x1 + c1 x2)
  Tn w1[3], b1[3], g1[3];
  w1[0] = v1 + wE0;
  w1[1] = tfmas(c1, wE1, s1 * wE2);
  w1[2] = tfmas(c1, wE2, s1 * (-wE1));
  b1[0] = tconst(aE0);
  b1[1] = tfma(w1[2], v1, tfmas(c1, aE1, s1 * aE2));   // + (w1 x e_x v1)_y = w1z v1
  b1[2] = tfma(w1[1], v1 * -1.f, tfmas(c1, aE2, s1 * (-aE1)));  // - w1y v1
  g1[0] = tconst(gE0);
  g1[1] = tfmas(c1, gE1, s1 * gE2);
  g1[2] = tfmas(c1, gE2, s1 * (-gE1));
  // box frame: R2^T x = (c2 x0 - s2 x2, x1, s2 x0 + c2 x2)
  Tn w2[3], b2[3], g2[3];
  w2[0] = c2 * w1[0] - s2 * w1[2];
  w2[1] = w1[1] + v2;
  w2[2] = tfma(s2, w1[0], c2 * w1[2]);
  b2[0] = c2 * b1[0] - s2 * b1[2] - w2[2] * v2;          // + (w2 x e_y v2)_x = -w2z v2
  b2[1] = b1[1];
  b2[2] = tfma(s2, b1[0], c2 * b1[2]) + w2[0] * v2;       // + w2x v2
  g2[0] = c2 * g1[0] - s2 * g1[2];
  g2[1] = g1[1];
  g2[2] = tfma(s2, g1[0], c2 * g1[2]);
  // bias moment Mb = I b2 + w2 x (I w2) + h x g2
  Tn Ib[3], Iw[3], Mb[3];
  Imul(bm, b2, Ib);
  Imul(bm, w2, Iw);
  Mb[0] = Ib[0] + (w2[1] * Iw[2] - w2[2] * Iw[1]) + (bm.h[1] * g2[2] - bm.h[2] * g2[1]);
  Mb[1] = Ib[1] + (w2[2] * Iw[0] - w2[0] * Iw[2]) + (bm.h[2] * g2[0] - bm.h[0] * g2[2]);
  Mb[2] = Ib[2] + (w2[0] * Iw[1] - w2[1] * Iw[0]) + (bm.h[0] * g2[1] - bm.h[1] * g2[0]);
  // joint axes in box coordinates: a1 = R2^T e_x = (c2, 0, s2), a2 = e_y
  Tn a1[3] = {c2, tconst(0.f), s2};
  Tn Ia1[3];
  Imul(bm, a1, Ia1);
  const Tn H11 = tfma(a1[0], Ia1[0], a1[2] * Ia1[2]);
  const Tn H12 = Ia1[1];
  const Tn H22 = bm.Iyy;
  const Tn r1 = v1 * (-ab.damping) - tfma(a1[0], Mb[0], a1[2] * Mb[2]);
  const Tn r2 = v2 * (-ab.damping) - Mb[1];
  const Tn det = H11 * H22 - H12 * H12;
  const Tn qdd1 = tdiv(H22 * r1 - H12 * r2, det);
  const Tn qdd2 = tdiv(H11 * r2 - H12 * r1, det);
  s[2] = tfmas(qdd1, dt, s[2]);
  s[3] = tfmas(qdd2, dt, s[3]);
  s[0] = tfmas(s[2], dt, s[0]);
  s[1] = tfmas(s[3], dt, s[1]);
}

template <bool FAST>
__global__ void __launch_bounds__(128) armbox_rollout_kernel(const ChainParams c, const ArmBoxParams ab,
                                                             const float* __restrict__ X, int N, Partials parts,
                                                             int grad, int32_t* __restrict__ status) {
  const size_t U = (size_t)N * c.W;
  const size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= U) return;
  const int w = (int)(u / N);
  const int i = (int)(u - (size_t)w * N);
  if (status && w == 0) status[i] = 0;
  float th[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) th[k] = __ldg(X + (size_t)k * N + i);
  const BoxMass bm = box_mass(ab, th);
  Tn s[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    s[k] = tconst(w == 0 ? c.s0[k] : __ldg(X + (size_t)(4 + (w - 1) * 4 + k) * N + i));
    if (w > 0) s[k].d[4 + k] = 1.f;
  }
  const int t0 = (int)(((long long)w * c.T) / c.W);
  const int t1 = (int)(((long long)(w + 1) * c.T) / c.W);
  float rss = 0.f;
  float g[kTan];
#pragma unroll
  for (int k = 0; k < kTan; ++k) g[k] = 0.f;
  for (int t = t0; t < t1; ++t) {
    box_step<FAST>(ab, bm, ab.base + (size_t)t * 9, c.dt, s);
    const float* row = c.obs + (size_t)t * c.D;  // observation x_{t+1}
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (c.obs_col[k] >= 0) {
        const float r = __ldg(row + c.obs_col[k]) - s[k].v;
        rss = fmaf(r, r, rss);
#pragma unroll
        for (int m = 0; m < kTan; ++m) g[m] = fmaf(r * c.inv_so2, s[k].d[m], g[m]);
      }
    }
  }
  float lp = -0.5f * c.inv_so2 * rss + (float)(t1 - t0) * c.obs_const;
  float nb[4] = {0.f, 0.f, 0.f, 0.f};
  if (w < c.W - 1) {
    const float* xs = X + (size_t)(4 + w * 4) * N + i;
    float dss = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float d = __ldg(xs + (size_t)k * N) - s[k].v;
      dss = fmaf(d, d, dss);
#pragma unroll
      for (int m = 0; m < kTan; ++m) g[m] = fmaf(d * c.inv_sd2, s[k].d[m], g[m]);
      nb[k] = -d * c.inv_sd2;
    }
    lp += -0.5f * c.inv_sd2 * dss + c.def_const;
  }
  parts.lp[(size_t)w * N + i] = lp;
  if (!grad) return;
  float* thp = parts.th + (size_t)w * 4 * N + i;
  float* st = parts.start + (size_t)w * 4 * N + i;
  float* nx = parts.next + (size_t)w * 4 * N + i;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    thp[(size_t)k * N] = g[k];
    st[(size_t)k * N] = g[4 + k];
    nx[(size_t)k * N] = nb[k];
  }
}

__global__ void __launch_bounds__(128) armbox_simulate_kernel(const ChainParams c, const ArmBoxParams ab,
                                                              const float* __restrict__ theta, int N,
                                                              float* __restrict__ states) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  float th[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) th[k] = theta[(size_t)k * N + i];
  const BoxMass bm = box_mass(ab, th);
  Tn s[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) s[k] = tconst(c.s0[k]);
  for (int t = 0; t <= c.T; ++t) {
    if (t > 0) box_step<false>(ab, bm, ab.base + (size_t)(t - 1) * 9, c.dt, s);
    float* out = states + (size_t)t * 4 * N + i;
#pragma unroll
    for (int k = 0; k < 4; ++k) out[(size_t)k * N] = s[k].v;
  }
}

cudaError_t launch_armbox_rollout(const ChainParams& c, const ArmBoxParams& ab, const float* X, int N,
                                  const Partials& parts, int grad, int32_t* status, cudaStream_t st) {
  const size_t U = (size_t)N * c.W;
  const unsigned blocks = (unsigned)((U + 127) / 128);
  if (c.fast_math)
    armbox_rollout_kernel<true><<<blocks, 128, 0, st>>>(c, ab, X, N, parts, grad, status);
  else
    armbox_rollout_kernel<false><<<blocks, 128, 0, st>>>(c, ab, X, N, parts, grad, status);
  return cudaGetLastError();
}

cudaError_t launch_armbox_simulate(const ChainParams& c, const ArmBoxParams& ab, const float* theta, int N,
                                   float* states, cudaStream_t st) {
  armbox_simulate_kernel<<<(N + 127) / 128, 128, 0, st>>>(c, ab, theta, N, states);
  return cudaGetLastError();
}

// ---- host: the arm's pivot motion, by classical kinematics in the world frame
namespace {
struct Vec3 {
  double x, y, z;
};
Vec3 operator+(Vec3 a, Vec3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
Vec3 operator-(Vec3 a, Vec3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
Vec3 operator*(Vec3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
Vec3 cross(Vec3 a, Vec3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
struct Mat3 {
  double m[3][3];
};
Mat3 matmul(const Mat3& a, const Mat3& b) {
  Mat3 r;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r.m[i][j] = a.m[i][0] * b.m[0][j] + a.m[i][1] * b.m[1][j] + a.m[i][2] * b.m[2][j];
  return r;
}
Vec3 apply(const Mat3& a, Vec3 v) {
  return {a.m[0][0] * v.x + a.m[0][1] * v.y + a.m[0][2] * v.z, a.m[1][0] * v.x + a.m[1][1] * v.y + a.m[1][2] * v.z,
          a.m[2][0] * v.x + a.m[2][1] * v.y + a.m[2][2] * v.z};
}
Vec3 apply_t(const Mat3& a, Vec3 v) {
  return {a.m[0][0] * v.x + a.m[1][0] * v.y + a.m[2][0] * v.z, a.m[0][1] * v.x + a.m[1][1] * v.y + a.m[2][1] * v.z,
          a.m[0][2] * v.x + a.m[1][2] * v.y + a.m[2][2] * v.z};
}
Mat3 rotation(int axis, double q) {  // active rotation about a principal axis
  const double c = cos(q), s = sin(q);
  Mat3 r{{{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}};
  const int i = (axis + 1) % 3, j = (axis + 2) % 3;
  r.m[i][i] = c;
  r.m[i][j] = -s;
  r.m[j][i] = s;
  r.m[j][j] = c;
  return r;
}
}  // namespace

// base[t] = (omega, alpha, a_pivot - g) of the pivot at time t*dt, in pivot coordinates
static void pivot_table(const pds_armbox_desc& d, double dt, int T, std::vector<float>& out) {
  out.assign((size_t)T * 9, 0.f);
  for (int t = 0; t < T; ++t) {
    const double time = t * dt;
    Mat3 R{{{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}};
    Vec3 w{0, 0, 0}, al{0, 0, 0}, v{0, 0, 0}, a{0, 0, 0};
    for (int j = 0; j < d.n_arm; ++j) {
      double q = 0, qd = 0, qdd = 0;
      for (int k = 0; k < 3; ++k) {
        const double A = d.amp[3 * j + k], om = 2.0 * M_PI * d.freq[3 * j + k], ph = d.phase[3 * j + k];
        q += A * sin(om * time + ph);
        qd += A * om * cos(om * time + ph);
        qdd += -A * om * om * sin(om * time + ph);
      }
      const int axis = (j % 2 == 0) ? 2 : 1;
      Vec3 e{0, 0, 0};
      if (axis == 2) e.z = 1; else e.y = 1;
      const Vec3 z = apply(R, e);  // joint axis in the world (unchanged by its own rotation)
      const Vec3 w_prev = w;
      w = w + z * qd;
      al = al + z * qdd + cross(w_prev, z * qd);
      R = matmul(R, rotation(axis, q));
      // move to the next joint (or the pivot) along the link's z axis
      const Vec3 r = apply(R, Vec3{0, 0, d.arm_len[j]});
      a = a + cross(al, r) + cross(w, cross(w, r));
      v = v + cross(w, r);
    }
    const Vec3 g{0, 0, -d.gravity};
    const Vec3 wl = apply_t(R, w), all = apply_t(R, al), ag = apply_t(R, a - g);
    float* o = out.data() + (size_t)t * 9;
    o[0] = (float)wl.x; o[1] = (float)wl.y; o[2] = (float)wl.z;
    o[3] = (float)all.x; o[4] = (float)all.y; o[5] = (float)all.z;
    o[6] = (float)ag.x; o[7] = (float)ag.y; o[8] = (float)ag.z;
  }
}

}  // namespace pds

using namespace pds;

extern "C" int pds_problem_create_armbox(const pds_armbox_desc* sys, double dt, int T, int windows, const float* obs,
                                         int D, const int* obs_index, double sigma_obs, double sigma_def,
                                         const float* s0, const float* theta_lo, const float* theta_hi, double c_lim,
                                         void* cuda_stream, pds_problem_t* out) {
  if (!out) return set_error(PDS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!sys || !sys->arm_len || !sys->amp || !sys->freq || !sys->phase)
    return set_error(PDS_ERR_ARG, "NULL arm description");
  if (sys->n_arm < 1 || sys->n_arm > PDS_MAX_LINKS) return set_error(PDS_ERR_UNSUPPORTED, "n_arm outside 1..8");
  if (!(sys->box_mass > 0) || !(sys->box_side > 0) || !(sys->weight_mass[0] >= 0) || !(sys->weight_mass[1] >= 0))
    return set_error(PDS_ERR_ARG, "bad box description");
  // Reuse the chain problem for validation and the common fields: a 2-link
  // "chain" with 4 theta entries gives n = 2, M = 4, S = 4 and the same
  // window layout; the dynamics fields are then replaced.
  const double ones[2] = {1.0, 1.0}, zeros[2] = {0.0, 0.0};
  const int kinds[4] = {PDS_PARAM_MASS, PDS_PARAM_MASS, PDS_PARAM_LENGTH, PDS_PARAM_LENGTH};
  const int links[4] = {0, 1, 0, 1};
  pds_system_desc chain;
  chain.kind = PDS_SYSTEM_PLANAR_CHAIN;
  chain.n_links = 2;
  chain.mass = ones;
  chain.length = ones;
  chain.damping = zeros;
  chain.gravity = sys->gravity;
  chain.n_theta = 4;
  chain.theta_kind = kinds;
  chain.theta_link = links;
  int rc = pds_problem_create(&chain, dt, T, windows, obs, D, obs_index, sigma_obs, sigma_def, s0, theta_lo, theta_hi,
                              c_lim, cuda_stream, out);
  if (rc != PDS_OK) return rc;
  pds_problem* p = *out;
  p->kind = PDS_SYSTEM_ARM_BOX;
  std::vector<float> table;
  pivot_table(*sys, dt, T, table);
  cudaError_t e = cudaMalloc(&p->d_base, table.size() * sizeof(float));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_base, table.data(), table.size() * sizeof(float), cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) {
    pds_problem_destroy(p);
    *out = nullptr;
    return set_error(PDS_ERR_CUDA, "arm-box: pivot table upload failed");
  }
  p->ab.box_mass = (float)sys->box_mass;
  p->ab.box_side = (float)sys->box_side;
  p->ab.box_com_depth = (float)sys->box_com_depth;
  p->ab.w_mass0 = (float)sys->weight_mass[0];
  p->ab.w_mass1 = (float)sys->weight_mass[1];
  p->ab.w_depth = (float)sys->weight_depth;
  p->ab.damping = (float)sys->damping;
  p->ab.base = p->d_base;
  return PDS_OK;
}
