// Rigid double pendulum with general inertia and centre of mass: the
// 11-parameter model of the physical double pendulum (Sec. V, real-world
// experiment; App. Table params-ibm-pendulum), rollout with its hand-written
// adjoint, simulation, and problem creation.
//
// Two rigid links on parallel revolute joints (axis z), joint 2 at (0, -l)
// in link 1's frame, gravity along -y.  Link k has mass m_k, centre of mass
// a_k = (akx, aky) in its frame and rotational inertia I_k about the COM
// axis; viscous joint friction -b_k qd_k.  With parallel axes the motion is
// planar, and the spatial equations reduce to the 2x2 system
//   M(q2) qdd = -b qd - C(q, qd) - G(q),
//   M11 = A + 2h, M12 = J2 + h, M22 = J2,  h = -(s2 Kx + c2 Ky),
//   C1 = hp qd2 (2 qd1 + qd2), C2 = -hp qd1^2,  hp = -(c2 Kx - s2 Ky),
//   G2 = c12 P2x - s12 P2y,  G1 = c1 P1x + s1 (Lg - P1y) + G2,
// with the per-particle constants
//   J2 = I2 + m2 |a2|^2,  A = I1 + m1 |a1|^2 + m2 l^2 + J2,
//   Kx,y = m2 l a2x,y,  P1x,y = g m1 a1x,y,  P2x,y = g m2 a2x,y,  Lg = g m2 l
// (s_k, c_k: sin, cos of q_k; s12, c12 of q1 + q2 by composition), solved in
// closed form; semi-implicit Euler as for the chains (App. B-A).
//
// Gradient: reverse mode.  The forward pass of a (particle, window) unit
// stores the state every K steps; the reverse sweep recomputes each segment's
// states and runs the adjoint of every step (the 2x2 solve's adjoint is
// z = M^-1 ybar, rbar = z, Mbar = -z y^T), accumulating the adjoints of the
// ten per-particle constants and the two friction coefficients, which map to
// the 11 parameters once per unit.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "pds_internal.cuh"

namespace pds {

namespace {

struct R2Const {
  float A, J2, Kx, Ky, P1x, P1y, Lg, P2x, P2y, b1, b2;
};

struct R2ConstBar {
  float A, J2, Kx, Ky, P1x, P1y, Lg, P2x, P2y, b1, b2;
};

__device__ __forceinline__ R2Const r2_constants(const float (&p)[kRigid2Params], float g) {
  const float m1 = p[0], I1 = p[1], a1x = p[2], a1y = p[3], l = p[5], m2 = p[6], I2 = p[7], a2x = p[8], a2y = p[9];
  R2Const k;
  k.J2 = fmaf(m2, fmaf(a2x, a2x, a2y * a2y), I2);
  k.A = I1 + m1 * fmaf(a1x, a1x, a1y * a1y) + m2 * l * l + k.J2;
  k.Kx = m2 * l * a2x;
  k.Ky = m2 * l * a2y;
  k.P1x = g * m1 * a1x;
  k.P1y = g * m1 * a1y;
  k.Lg = g * m2 * l;
  k.P2x = g * m2 * a2x;
  k.P2y = g * m2 * a2y;
  k.b1 = p[4];
  k.b2 = p[10];
  return k;
}

// Intermediates of one step from state s.
struct R2Fwd {
  float s1, c1, s2, c2, s12, c12, h, hp, M11, M12, M22, idet, y1, y2;
};

template <bool FAST>
__device__ __forceinline__ R2Fwd r2_forward(const R2Const& k, const float (&s)[4]) {
  R2Fwd f;
  if (FAST) {
    __sincosf(s[0], &f.s1, &f.c1);
    __sincosf(s[1], &f.s2, &f.c2);
  } else {
    sincosf(s[0], &f.s1, &f.c1);
    sincosf(s[1], &f.s2, &f.c2);
  }
  f.s12 = fmaf(f.s1, f.c2, f.c1 * f.s2);
  f.c12 = fmaf(f.c1, f.c2, -f.s1 * f.s2);
  f.h = -fmaf(f.s2, k.Kx, f.c2 * k.Ky);
  f.hp = -fmaf(f.c2, k.Kx, -f.s2 * k.Ky);
  f.M11 = fmaf(2.f, f.h, k.A);
  f.M12 = k.J2 + f.h;
  f.M22 = k.J2;
  const float v1 = s[2], v2 = s[3];
  const float G2 = fmaf(f.c12, k.P2x, -f.s12 * k.P2y);
  const float G1 = fmaf(f.c1, k.P1x, fmaf(f.s1, k.Lg - k.P1y, G2));
  const float r1 = -fmaf(k.b1, v1, fmaf(f.hp * v2, fmaf(2.f, v1, v2), G1));
  const float r2 = fmaf(f.hp * v1, v1, -fmaf(k.b2, v2, G2));
  const float det = fmaf(f.M11, f.M22, -f.M12 * f.M12);
  f.idet = FAST ? __frcp_rn(det) : 1.0f / det;
  f.y1 = fmaf(f.M22, r1, -f.M12 * r2) * f.idet;
  f.y2 = fmaf(f.M11, r2, -f.M12 * r1) * f.idet;
  return f;
}

__device__ __forceinline__ void r2_apply(const R2Fwd& f, float dt, float (&s)[4]) {
  s[2] = fmaf(dt, f.y1, s[2]);
  s[3] = fmaf(dt, f.y2, s[3]);
  s[0] = fmaf(dt, s[2], s[0]);
  s[1] = fmaf(dt, s[3], s[1]);
}

// Adjoint of one step: a holds the adjoint of the state after the step on
// entry and of the state s before it on return; kb accumulates the
// constants' adjoints.
__device__ __forceinline__ void r2_reverse(const R2Const& k, const R2Fwd& f, const float (&s)[4], float dt,
                                           float (&a)[4], R2ConstBar& kb) {
  const float v1 = s[2], v2 = s[3];
  const float W1 = fmaf(dt, a[0], a[2]), W2 = fmaf(dt, a[1], a[3]);  // adjoints of v1', v2'
  const float Y1 = dt * W1, Y2 = dt * W2;
  const float z1 = fmaf(f.M22, Y1, -f.M12 * Y2) * f.idet;
  const float z2 = fmaf(f.M11, Y2, -f.M12 * Y1) * f.idet;
  const float Mb11 = -z1 * f.y1, Mb22 = -z2 * f.y2, Mb12 = -fmaf(z1, f.y2, z2 * f.y1);
  // r1 = -b1 v1 - hp v2 (2 v1 + v2) - G1;  r2 = -b2 v2 + hp v1^2 - G2
  const float vb1 = W1 + z1 * fmaf(-2.f * f.hp, v2, -k.b1) + z2 * (2.f * f.hp * v1);
  const float vb2 = W2 - z1 * (2.f * f.hp * (v1 + v2)) - z2 * k.b2;
  kb.b1 = fmaf(-z1, v1, kb.b1);
  kb.b2 = fmaf(-z2, v2, kb.b2);
  const float hpb = fmaf(z2, v1 * v1, -z1 * v2 * fmaf(2.f, v1, v2));
  const float G1b = -z1, G2b = -z2 + G1b;
  // G1 = c1 P1x + s1 (Lg - P1y) + G2
  float c1b = G1b * k.P1x, s1b = G1b * (k.Lg - k.P1y);
  kb.P1x = fmaf(G1b, f.c1, kb.P1x);
  kb.Lg = fmaf(G1b, f.s1, kb.Lg);
  kb.P1y = fmaf(-G1b, f.s1, kb.P1y);
  // G2 = c12 P2x - s12 P2y
  const float c12b = G2b * k.P2x, s12b = -G2b * k.P2y;
  kb.P2x = fmaf(G2b, f.c12, kb.P2x);
  kb.P2y = fmaf(-G2b, f.s12, kb.P2y);
  // s12 = s1 c2 + c1 s2, c12 = c1 c2 - s1 s2
  s1b += fmaf(s12b, f.c2, -c12b * f.s2);
  c1b += fmaf(s12b, f.s2, c12b * f.c2);
  float s2b = fmaf(s12b, f.c1, -c12b * f.s1);
  float c2b = fmaf(s12b, f.s1, c12b * f.c1);
  // M11 = A + 2h, M12 = J2 + h, M22 = J2
  kb.A += Mb11;
  kb.J2 += Mb12 + Mb22;
  const float hb = fmaf(2.f, Mb11, Mb12);
  // h = -(s2 Kx + c2 Ky), hp = -(c2 Kx - s2 Ky)
  s2b += fmaf(-hb, k.Kx, hpb * k.Ky);
  c2b += fmaf(-hb, k.Ky, -hpb * k.Kx);
  kb.Kx += fmaf(-hb, f.s2, -hpb * f.c2);
  kb.Ky += fmaf(-hb, f.c2, hpb * f.s2);
  a[0] += fmaf(s1b, f.c1, -c1b * f.s1);
  a[1] += fmaf(s2b, f.c2, -c2b * f.s2);
  a[2] = vb1;
  a[3] = vb2;
}

// Parameter adjoints from the constants' adjoints.
__device__ __forceinline__ void r2_param_grad(const float (&p)[kRigid2Params], float g, const R2ConstBar& kb,
                                              float (&pb)[kRigid2Params]) {
  const float m1 = p[0], a1x = p[2], a1y = p[3], l = p[5], m2 = p[6], a2x = p[8], a2y = p[9];
  const float J2b = kb.J2 + kb.A;
  pb[0] = kb.A * fmaf(a1x, a1x, a1y * a1y) + g * fmaf(kb.P1x, a1x, kb.P1y * a1y);
  pb[1] = kb.A;
  pb[2] = 2.f * kb.A * m1 * a1x + kb.P1x * g * m1;
  pb[3] = 2.f * kb.A * m1 * a1y + kb.P1y * g * m1;
  pb[4] = kb.b1;
  pb[5] = 2.f * kb.A * m2 * l + kb.Lg * g * m2 + m2 * fmaf(kb.Kx, a2x, kb.Ky * a2y);
  pb[6] = kb.A * l * l + J2b * fmaf(a2x, a2x, a2y * a2y) + g * (kb.Lg * l + fmaf(kb.P2x, a2x, kb.P2y * a2y)) +
          l * fmaf(kb.Kx, a2x, kb.Ky * a2y);
  pb[7] = J2b;
  pb[8] = 2.f * J2b * m2 * a2x + kb.P2x * g * m2 + kb.Kx * m2 * l;
  pb[9] = 2.f * J2b * m2 * a2y + kb.P2y * g * m2 + kb.Ky * m2 * l;
  pb[10] = kb.b2;
}

__device__ __forceinline__ void load_rigid2_params(const Rigid2Params& r, const float* __restrict__ X, int N, int i,
                                                   float (&p)[kRigid2Params]) {
#pragma unroll
  for (int k = 0; k < kRigid2Params; ++k)
    p[k] = r.theta_row[k] >= 0 ? __ldg(X + (size_t)r.theta_row[k] * N + i) : r.p[k];
}

// Observation residual of row t (the observation of the state after step t)
// against state x: returns r^2 summed over the observed components and, if
// seed, adds r / sigma^2 to a.  EVERY (all four components observed): one
// 16-byte load of the state-ordered row, no per-component test; otherwise
// each component looks up its column.
template <bool EVERY>
__device__ __forceinline__ float r2_residual(const ChainParams& c, int t, const float (&x)[4], float (&a)[4],
                                             bool seed) {
  float acc = 0.f;
  if constexpr (EVERY) {
    const float4 o = __ldg(reinterpret_cast<const float4*>(c.obs_s) + t);
    const float e[4] = {o.x - x[0], o.y - x[1], o.z - x[2], o.w - x[3]};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      acc = fmaf(e[q], e[q], acc);
      if (seed) a[q] = fmaf(c.inv_so2, e[q], a[q]);
    }
  } else {
    const float* row = c.obs + (size_t)t * c.D;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (c.obs_col[q] >= 0) {
        const float e = __ldg(row + c.obs_col[q]) - x[q];
        acc = fmaf(e, e, acc);
        if (seed) a[q] = fmaf(c.inv_so2, e, a[q]);
      }
  }
  return acc;
}

}  // namespace

// The checkpoint tape is thread-contiguous, [slot][U] of float4 (one 16-byte
// access per state); the K > 1 segment buffer stays [K][4][U].
template <bool FAST, bool EVERY>
__global__ void __launch_bounds__(128) rigid2_rollout_kernel(const ChainParams c, const Rigid2Params r,
                                                             const float* __restrict__ X, int N, Partials parts,
                                                             int grad, int32_t* __restrict__ status) {
  const size_t U = (size_t)N * c.W;
  const size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= U) return;
  const int w = (int)(u / N);
  const int i = (int)(u - (size_t)w * N);
  if (status && w == 0) status[i] = 0;
  float p[kRigid2Params];
  load_rigid2_params(r, X, N, i, p);
  const R2Const k = r2_constants(p, c.g);
  float s[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) s[q] = w == 0 ? c.s0[q] : __ldg(X + (size_t)(c.M + (w - 1) * 4 + q) * N + i);
  const int t0 = (int)(((long long)w * c.T) / c.W);
  const int t1 = (int)(((long long)(w + 1) * c.T) / c.W);
  const int K = c.K;
  float4* ck = reinterpret_cast<float4*>(parts.tape);     // [max_seg][U]
  float* seg = parts.tape + (size_t)c.max_seg * 4 * U;     // [K][4][U]
  float rss = 0.f;
  float unused[4];
  int kk = 0, slot = 0;  // step within the checkpoint stride, checkpoint slot
  for (int t = t0; t < t1; ++t) {
    if (grad && kk == 0) ck[(size_t)slot * U + u] = make_float4(s[0], s[1], s[2], s[3]);
    if (++kk == K) {
      kk = 0;
      ++slot;
    }
    const R2Fwd f = r2_forward<FAST>(k, s);
    r2_apply(f, c.dt, s);
    rss += r2_residual<EVERY>(c, t, s, unused, false);  // observation x_{t+1}
  }
  float lp = -0.5f * c.inv_so2 * rss + (float)(t1 - t0) * c.obs_const;
  float a[4] = {0.f, 0.f, 0.f, 0.f};
  float nb[4] = {0.f, 0.f, 0.f, 0.f};
  if (w < c.W - 1) {
    const float* xs = X + (size_t)(c.M + w * 4) * N + i;
    float dss = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float d = __ldg(xs + (size_t)q * N) - s[q];
      dss = fmaf(d, d, dss);
      a[q] = d * c.inv_sd2;
      nb[q] = -d * c.inv_sd2;
    }
    lp += -0.5f * c.inv_sd2 * dss + c.def_const;
  }
  parts.lp[(size_t)w * N + i] = lp;
  if (!grad) return;
  R2ConstBar kb;
  kb.A = kb.J2 = kb.Kx = kb.Ky = kb.P1x = kb.P1y = kb.Lg = kb.P2x = kb.P2y = kb.b1 = kb.b2 = 0.f;
  const int h = t1 - t0;
  if (K == 1) {
    // every pre-step state is on the tape; the state of step j-1 is loaded
    // while step j is reversed
    float x[4], xn[4] = {0.f, 0.f, 0.f, 0.f};
    float4 v4 = ck[(size_t)(h - 1) * U + u];
    x[0] = v4.x; x[1] = v4.y; x[2] = v4.z; x[3] = v4.w;
    for (int j = h - 1; j >= 0; --j) {
      if (j > 0) {
        v4 = ck[(size_t)(j - 1) * U + u];
        xn[0] = v4.x; xn[1] = v4.y; xn[2] = v4.z; xn[3] = v4.w;
      }
      const R2Fwd f = r2_forward<FAST>(k, x);
      float xa[4] = {x[0], x[1], x[2], x[3]};
      r2_apply(f, c.dt, xa);
      r2_residual<EVERY>(c, t0 + j, xa, a, true);
      r2_reverse(k, f, x, c.dt, a, kb);
#pragma unroll
      for (int q = 0; q < 4; ++q) x[q] = xn[q];
    }
  }
  const int nseg = K == 1 ? 0 : (h + K - 1) / K;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int ta = sg * K, tb = min(h, ta + K);
    // recompute the segment's pre-step states
    const float4 v4 = ck[(size_t)sg * U + u];
    float x[4] = {v4.x, v4.y, v4.z, v4.w};
    for (int j = 0; j < tb - ta; ++j) {
      float* o = seg + (size_t)j * 4 * U + u;
#pragma unroll
      for (int q = 0; q < 4; ++q) o[(size_t)q * U] = x[q];
      if (j + 1 < tb - ta) {
        const R2Fwd f = r2_forward<FAST>(k, x);
        r2_apply(f, c.dt, x);
      }
    }
    for (int j = tb - ta - 1; j >= 0; --j) {
      const float* o = seg + (size_t)j * 4 * U + u;
#pragma unroll
      for (int q = 0; q < 4; ++q) x[q] = o[(size_t)q * U];
      const R2Fwd f = r2_forward<FAST>(k, x);
      float xn[4] = {x[0], x[1], x[2], x[3]};
      r2_apply(f, c.dt, xn);
      // observation seed of the state after the step
      r2_residual<EVERY>(c, t0 + ta + j, xn, a, true);
      r2_reverse(k, f, x, c.dt, a, kb);
    }
  }
  float pb[kRigid2Params];
  r2_param_grad(p, c.g, kb, pb);
  float* thp = parts.th + (size_t)w * c.M * N + i;
#pragma unroll
  for (int q = 0; q < kRigid2Params; ++q)
    if (r.theta_row[q] >= 0) thp[(size_t)r.theta_row[q] * N] = pb[q];
  float* st = parts.start + (size_t)w * 4 * N + i;
  float* nx = parts.next + (size_t)w * 4 * N + i;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    st[(size_t)q * N] = a[q];
    nx[(size_t)q * N] = nb[q];
  }
}

__global__ void __launch_bounds__(128) rigid2_simulate_kernel(const ChainParams c, const Rigid2Params r,
                                                              const float* __restrict__ theta, int N,
                                                              float* __restrict__ states) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  float p[kRigid2Params];
#pragma unroll
  for (int k = 0; k < kRigid2Params; ++k) p[k] = r.theta_row[k] >= 0 ? theta[(size_t)r.theta_row[k] * N + i] : r.p[k];
  const R2Const kc = r2_constants(p, c.g);
  float s[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) s[q] = c.s0[q];
  for (int t = 0; t <= c.T; ++t) {
    if (t > 0) {
      const R2Fwd f = r2_forward<false>(kc, s);
      r2_apply(f, c.dt, s);
    }
    float* out = states + (size_t)t * 4 * N + i;
#pragma unroll
    for (int q = 0; q < 4; ++q) out[(size_t)q * N] = s[q];
  }
}

cudaError_t launch_rigid2_rollout(const ChainParams& c, const Rigid2Params& r, const float* X, int N,
                                  const Partials& parts, int grad, int32_t* status, cudaStream_t st) {
  const size_t U = (size_t)N * c.W;
  const unsigned blocks = (unsigned)((U + 127) / 128);
  const bool every = (c.obs_mask & 0xFu) == 0xFu;
  if (c.fast_math && every)
    rigid2_rollout_kernel<true, true><<<blocks, 128, 0, st>>>(c, r, X, N, parts, grad, status);
  else if (c.fast_math)
    rigid2_rollout_kernel<true, false><<<blocks, 128, 0, st>>>(c, r, X, N, parts, grad, status);
  else if (every)
    rigid2_rollout_kernel<false, true><<<blocks, 128, 0, st>>>(c, r, X, N, parts, grad, status);
  else
    rigid2_rollout_kernel<false, false><<<blocks, 128, 0, st>>>(c, r, X, N, parts, grad, status);
  return cudaGetLastError();
}

cudaError_t launch_rigid2_simulate(const ChainParams& c, const Rigid2Params& r, const float* theta, int N,
                                   float* states, cudaStream_t st) {
  rigid2_simulate_kernel<<<(N + 127) / 128, 128, 0, st>>>(c, r, theta, N, states);
  return cudaGetLastError();
}

}  // namespace pds

using namespace pds;

extern "C" int pds_problem_create_rigid2(const pds_rigid2_desc* sys, double dt, int T, int windows, const float* obs,
                                         int D, const int* obs_index, double sigma_obs, double sigma_def,
                                         const float* s0, const float* theta_lo, const float* theta_hi, double c_lim,
                                         void* cuda_stream, pds_problem_t* out) {
  if (!out) return set_error(PDS_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!sys || !sys->theta_param || !theta_lo || !theta_hi) return set_error(PDS_ERR_ARG, "NULL argument");
  const int M = sys->n_theta;
  if (M < 1 || M > kRigid2Params) return set_error(PDS_ERR_ARG, "n_theta outside 1..11");
  int row_of[kRigid2Params];
  for (int k = 0; k < kRigid2Params; ++k) row_of[k] = -1;
  for (int k = 0; k < M; ++k) {
    const int q = sys->theta_param[k];
    if (q < 0 || q >= kRigid2Params) return set_error(PDS_ERR_ARG, "theta_param entry outside 0..10");
    if (row_of[q] >= 0) return set_error(PDS_ERR_ARG, "theta_param repeats a parameter");
    row_of[q] = k;
    if (!(theta_hi[k] > theta_lo[k])) return set_error(PDS_ERR_ARG, "empty theta box");
  }
  // The chain problem validates and stores the common fields: a 2-link chain
  // gives n = 2, S = 4 and the window layout; M, the box and the dynamics
  // are then replaced.
  const double ones[2] = {1.0, 1.0}, zeros[2] = {0.0, 0.0};
  const int kinds[1] = {PDS_PARAM_MASS};
  const int links[1] = {0};
  pds_system_desc chain;
  chain.kind = PDS_SYSTEM_PLANAR_CHAIN;
  chain.n_links = 2;
  chain.mass = ones;
  chain.length = ones;
  chain.damping = zeros;
  chain.gravity = sys->gravity;
  chain.n_theta = 1;
  chain.theta_kind = kinds;
  chain.theta_link = links;
  int rc = pds_problem_create(&chain, dt, T, windows, obs, D, obs_index, sigma_obs, sigma_def, s0, theta_lo, theta_hi,
                              c_lim, cuda_stream, out);
  if (rc != PDS_OK) return rc;
  pds_problem* p = *out;
  p->kind = PDS_SYSTEM_RIGID_DOUBLE_PENDULUM;
  ChainParams& c = p->c;
  c.M = M;
  c.P = M + (windows - 1) * 4;
  double lim = 0.0;
  for (int k = 0; k < M; ++k) {
    c.lo[k] = theta_lo[k];
    c.hi[k] = theta_hi[k];
    lim -= log((double)theta_hi[k] - (double)theta_lo[k]);
  }
  c.lim_const = (float)lim;
  c.mass_theta[0] = -1;
  for (int k = 0; k < kRigid2Params; ++k) {
    p->r2.p[k] = (float)sys->param[k];
    p->r2.theta_row[k] = row_of[k];
    p->r2.theta_param[k] = k < M ? sys->theta_param[k] : 0;
  }
  return PDS_OK;
}
