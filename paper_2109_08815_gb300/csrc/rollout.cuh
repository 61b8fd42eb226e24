// Fused window rollout + hand-written reverse adjoint for planar point-mass
// chains (one thread per particle-window unit).
//
// Forward dynamics (Appendix B-A, Eq. dynamics): the articulated-body
// recursion specialised to a planar chain whose links are massless rods with
// a point mass at the tip.  Every frame is world-aligned and sits at the
// joint, so the joint motion subspace is (1, 0, 0) and the articulated
// inertia passed from link i to its parent has only a 2x2 translational
// block K (a revolute joint transmits no moment).  With
//   r_i   = l_i (sin phi_i, -cos phi_i)   link vector p_i - p_{i-1}
//   rho_i = l_i (cos phi_i,  sin phi_i)   its derivative d r_i / d phi_i
//   phi_i = q_1 + .. + q_i, omega_i = qd_1 + .. + qd_i  (absolute angle, rate)
// the inward pass (i = n..1, K_{n+1} = 0, B_{n+1} = 0, tau_{n+1} = 0) is
//   A_i = K_{i+1} + m_i I,  Y_i = A_i rho_i,  D_i = rho_i . Y_i,
//   beta_i = B_{i+1} + m_i g e_y - omega_i^2 A_i r_i,
//   t_i = (tau_i - tau_{i+1} - rho_i . beta_i) / D_i,
//   B_i = beta_i + t_i Y_i,  K_i = A_i - Y_i Y_i^T / D_i,
// where the force link i's parent applies at joint i is K_i a_{i-1} + B_i
// (a_{i-1} = acceleration of joint i).  The outward pass (a_0 = 0) gives the
// absolute angular accelerations
//   alpha_i = t_i - Y_i . a_{i-1} / D_i,  a_i = a_{i-1} - omega_i^2 r_i + alpha_i rho_i,
// and qdd_i = alpha_i - alpha_{i-1}.  Semi-implicit Euler then updates
// qd += qdd dt, q += qd dt (the new velocity).
//
// The adjoint of one step is the exact reverse-mode derivative of the same
// arithmetic (Appendix B-A: gradients through f_step by the chain rule /
// adjoint method), written by hand statement by statement in reverse order.
#pragma once

#include "pds_internal.cuh"

#ifndef PDS_ROLLOUT_MINB
#define PDS_ROLLOUT_MINB 3
#endif

namespace pds {

// sin/cos and reciprocal: CUDA's accurate functions, or (FAST) the hardware
// approximations __sincosf / __fdividef, which the parity tests also cover.
template <bool FAST>
__device__ __forceinline__ void sc(float x, float* s, float* c) {
  if (FAST) __sincosf(x, s, c);
  else sincosf(x, s, c);
}
template <bool FAST>
__device__ __forceinline__ float rcp(float x) {
  return FAST ? __fdividef(1.0f, x) : 1.0f / x;
}

// Forward step in place.
template <int NL, bool FAST>
__device__ __forceinline__ void chain_step(float (&q)[NL], float (&v)[NL], const float (&m)[NL],
                                           const float (&l)[NL], const float (&b)[NL], float g, float dt) {
  float sn[NL], cs[NL], w2[NL], tau[NL];
  {
    float phi = 0.f, om = 0.f;
#pragma unroll
    for (int i = 0; i < NL; ++i) {
      phi += q[i];
      om += v[i];
      sc<FAST>(phi, &sn[i], &cs[i]);
      w2[i] = om * om;
      tau[i] = -b[i] * v[i];
    }
  }
  float Yx[NL], Yy[NL], iD[NL], tt[NL];
  float Kxx = 0.f, Kxy = 0.f, Kyy = 0.f, Bx = 0.f, By = 0.f, tnext = 0.f;
#pragma unroll
  for (int i = NL - 1; i >= 0; --i) {
    const float rx = l[i] * sn[i], ry = -l[i] * cs[i];
    const float px = l[i] * cs[i], py = l[i] * sn[i];
    const float Axx = Kxx + m[i], Axy = Kxy, Ayy = Kyy + m[i];
    const float yx = Axx * px + Axy * py, yy = Axy * px + Ayy * py;
    const float D = px * yx + py * yy;
    const float zx = Axx * rx + Axy * ry, zy = Axy * rx + Ayy * ry;
    const float bx = Bx - w2[i] * zx, by = By + m[i] * g - w2[i] * zy;
    const float id = rcp<FAST>(D);
    const float t = (tau[i] - tnext - (px * bx + py * by)) * id;
    Bx = bx + t * yx;
    By = by + t * yy;
    Kxx = Axx - yx * yx * id;
    Kxy = Axy - yx * yy * id;
    Kyy = Ayy - yy * yy * id;
    tnext = tau[i];
    Yx[i] = yx; Yy[i] = yy; iD[i] = id; tt[i] = t;
  }
  float ax = 0.f, ay = 0.f, aprev = 0.f;
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    const float al = tt[i] - (Yx[i] * ax + Yy[i] * ay) * iD[i];
    const float rx = l[i] * sn[i], ry = -l[i] * cs[i];
    const float px = l[i] * cs[i], py = l[i] * sn[i];
    ax = ax - w2[i] * rx + al * px;
    ay = ay - w2[i] * ry + al * py;
    const float qdd = al - aprev;
    aprev = al;
    v[i] = v[i] + qdd * dt;
    q[i] = q[i] + v[i] * dt;
  }
}

// Reverse of one step.  On entry (qb, vb) is the adjoint of the step's
// output state; on exit it is the adjoint of the input state (q, v).  The
// adjoints of the link parameters are accumulated into mb, lb, bb.
template <int NL, bool FAST>
__device__ __forceinline__ void chain_step_vjp(const float (&q)[NL], const float (&v)[NL], const float (&m)[NL],
                                               const float (&l)[NL], const float (&b)[NL], float g, float dt,
                                               float (&qb)[NL], float (&vb)[NL], float (&mb)[NL], float (&lb)[NL],
                                               float (&bb)[NL]) {
  // ---- recompute the forward intermediates at (q, v)
  float sn[NL], cs[NL], om[NL], tau[NL];
  {
    float phi = 0.f, o = 0.f;
#pragma unroll
    for (int i = 0; i < NL; ++i) {
      phi += q[i];
      o += v[i];
      sc<FAST>(phi, &sn[i], &cs[i]);
      om[i] = o;
      tau[i] = -b[i] * v[i];
    }
  }
  float Axx[NL], Axy[NL], Ayy[NL], iD[NL], bx[NL], by[NL], tt[NL], al[NL], a0x[NL], a0y[NL];
  {
    float Kxx = 0.f, Kxy = 0.f, Kyy = 0.f, Bx = 0.f, By = 0.f, tnext = 0.f;
#pragma unroll
    for (int i = NL - 1; i >= 0; --i) {
      const float rx = l[i] * sn[i], ry = -l[i] * cs[i];
      const float px = l[i] * cs[i], py = l[i] * sn[i];
      Axx[i] = Kxx + m[i]; Axy[i] = Kxy; Ayy[i] = Kyy + m[i];
      const float yx = Axx[i] * px + Axy[i] * py, yy = Axy[i] * px + Ayy[i] * py;
      const float D = px * yx + py * yy;
      const float zx = Axx[i] * rx + Axy[i] * ry, zy = Axy[i] * rx + Ayy[i] * ry;
      const float w2 = om[i] * om[i];
      bx[i] = Bx - w2 * zx;
      by[i] = By + m[i] * g - w2 * zy;
      iD[i] = rcp<FAST>(D);
      tt[i] = (tau[i] - tnext - (px * bx[i] + py * by[i])) * iD[i];
      Bx = bx[i] + tt[i] * yx;
      By = by[i] + tt[i] * yy;
      Kxx = Axx[i] - yx * yx * iD[i];
      Kxy = Axy[i] - yx * yy * iD[i];
      Kyy = Ayy[i] - yy * yy * iD[i];
      tnext = tau[i];
    }
    float ax = 0.f, ay = 0.f;
#pragma unroll
    for (int i = 0; i < NL; ++i) {
      const float rx = l[i] * sn[i], ry = -l[i] * cs[i];
      const float px = l[i] * cs[i], py = l[i] * sn[i];
      const float yx = Axx[i] * px + Axy[i] * py, yy = Axy[i] * px + Ayy[i] * py;
      a0x[i] = ax; a0y[i] = ay;
      al[i] = tt[i] - (yx * ax + yy * ay) * iD[i];
      const float w2 = om[i] * om[i];
      ax = ax - w2 * rx + al[i] * px;
      ay = ay - w2 * ry + al[i] * py;
    }
  }

  // ---- Euler: qd' = qd + qdd dt, q' = q + qd' dt
  float alb[NL];
#pragma unroll
  for (int i = 0; i < NL; ++i) vb[i] += qb[i] * dt;  // qb passes through unchanged
  // qdd_i = alpha_i - alpha_{i-1}  =>  alpha_i receives qdd_b[i] - qdd_b[i+1]
#pragma unroll
  for (int i = 0; i < NL; ++i) alb[i] = (vb[i] - ((i + 1 < NL) ? vb[i + 1] : 0.f)) * dt;

  // ---- reverse of the outward pass
  float rxb[NL], ryb[NL], pxb[NL], pyb[NL], omb[NL], tb[NL], Yxb[NL], Yyb[NL], Db[NL];
  {
    float axb = 0.f, ayb = 0.f;
#pragma unroll
    for (int i = NL - 1; i >= 0; --i) {
      const float rx = l[i] * sn[i], ry = -l[i] * cs[i];
      const float px = l[i] * cs[i], py = l[i] * sn[i];
      const float w2 = om[i] * om[i];
      // a_i = a_{i-1} - w2 r + alpha rho
      omb[i] = -2.f * om[i] * (rx * axb + ry * ayb);
      rxb[i] = -w2 * axb;
      ryb[i] = -w2 * ayb;
      alb[i] += px * axb + py * ayb;
      pxb[i] = al[i] * axb;
      pyb[i] = al[i] * ayb;
      // alpha_i = t_i - (Y . a_{i-1}) / D
      const float yx = Axx[i] * px + Axy[i] * py, yy = Axy[i] * px + Ayy[i] * py;
      tb[i] = alb[i];
      const float f = alb[i] * iD[i];
      Yxb[i] = -f * a0x[i];
      Yyb[i] = -f * a0y[i];
      Db[i] = f * (yx * a0x[i] + yy * a0y[i]) * iD[i];
      axb -= f * yx;
      ayb -= f * yy;
    }
  }

  // ---- reverse of the inward pass (parent to child)
  float taub[NL];
#pragma unroll
  for (int i = 0; i < NL; ++i) taub[i] = 0.f;
  {
    float Kxxb = 0.f, Kxyb = 0.f, Kyyb = 0.f, Bxb = 0.f, Byb = 0.f;
#pragma unroll
    for (int i = 0; i < NL; ++i) {
      const float rx = l[i] * sn[i], ry = -l[i] * cs[i];
      const float px = l[i] * cs[i], py = l[i] * sn[i];
      const float yx = Axx[i] * px + Axy[i] * py, yy = Axy[i] * px + Ayy[i] * py;
      const float zx = Axx[i] * rx + Axy[i] * ry, zy = Axy[i] * rx + Ayy[i] * ry;
      const float id = iD[i];
      const float w2 = om[i] * om[i];
      // K_i = A - Y Y^T / D
      float Axxb = Kxxb, Axyb = Kxyb, Ayyb = Kyyb;
      float yxb = Yxb[i] - (2.f * Kxxb * yx + Kxyb * yy) * id;
      float yyb = Yyb[i] - (Kxyb * yx + 2.f * Kyyb * yy) * id;
      float Dbar = Db[i] + (Kxxb * yx * yx + Kxyb * yx * yy + Kyyb * yy * yy) * id * id;
      // B_i = beta + t Y
      float bxb = Bxb, byb = Byb;
      const float tbar = tb[i] + Bxb * yx + Byb * yy;
      yxb += tt[i] * Bxb;
      yyb += tt[i] * Byb;
      // t = (tau_i - tau_{i+1} - rho . beta) / D
      const float ft = tbar * id;
      taub[i] += ft;
      if (i + 1 < NL) taub[i + 1] -= ft;
      float pxbar = pxb[i] - ft * bx[i];
      float pybar = pyb[i] - ft * by[i];
      bxb -= ft * px;
      byb -= ft * py;
      Dbar -= ft * tt[i];
      // beta = B_{i+1} + m g e_y - w2 Z
      mb[i] += g * byb;
      float ombar = omb[i] - 2.f * om[i] * (zx * bxb + zy * byb);
      const float zxb = -w2 * bxb, zyb = -w2 * byb;
      // Z = A r
      Axxb += zxb * rx;
      Axyb += zxb * ry + zyb * rx;
      Ayyb += zyb * ry;
      float rxbar = rxb[i] + Axx[i] * zxb + Axy[i] * zyb;
      float rybar = ryb[i] + Axy[i] * zxb + Ayy[i] * zyb;
      // D = rho . Y
      pxbar += Dbar * yx;
      pybar += Dbar * yy;
      yxb += Dbar * px;
      yyb += Dbar * py;
      // Y = A rho
      Axxb += yxb * px;
      Axyb += yxb * py + yyb * px;
      Ayyb += yyb * py;
      pxbar += Axx[i] * yxb + Axy[i] * yyb;
      pybar += Axy[i] * yxb + Ayy[i] * yyb;
      // A = K_{i+1} + m I
      mb[i] += Axxb + Ayyb;
      Kxxb = Axxb; Kxyb = Axyb; Kyyb = Ayyb;
      Bxb = bxb; Byb = byb;
      // kinematics: r = l (s, -c), rho = l (c, s); d r / d phi = rho, d rho / d phi = -r
      const float phib = rxbar * px + rybar * py - (pxbar * rx + pybar * ry);
      lb[i] += rxbar * sn[i] - rybar * cs[i] + pxbar * cs[i] + pybar * sn[i];
      // stash phi / omega adjoints in rxb / ryb for the prefix-sum reverse
      rxb[i] = phib;
      ryb[i] = ombar;
    }
  }
  // tau_i = -b_i v_i ; phi_i = sum_{j<=i} q_j ; omega_i = sum_{j<=i} v_j
  float sphi = 0.f, som = 0.f;
#pragma unroll
  for (int i = NL - 1; i >= 0; --i) {
    sphi += rxb[i];
    som += ryb[i];
    bb[i] += -taub[i] * v[i];
    qb[i] += sphi;
    vb[i] += som - taub[i] * b[i];
  }
}

// Load the physical parameters of particle i (defaults overridden by theta).
template <int NL>
__device__ __forceinline__ void load_params(const ChainParams& c, const float* __restrict__ X, int N, int i,
                                            float (&m)[NL], float (&l)[NL], float (&b)[NL]) {
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    m[j] = (c.mass_theta[j] >= 0) ? __ldg(X + (size_t)c.mass_theta[j] * N + i) : c.mass[j];
    l[j] = (c.length_theta[j] >= 0) ? __ldg(X + (size_t)c.length_theta[j] * N + i) : c.length[j];
    b[j] = (c.damp_theta[j] >= 0) ? __ldg(X + (size_t)c.damp_theta[j] * N + i) : c.damping[j];
  }
}

// Observation residual terms of one step: returns sum of r^2 over observed
// components of state (q, v) at time t (1-based), and if seed != nullptr adds
// d/ds [-r^2 / (2 sigma^2)] = r / sigma^2 to the state adjoint.
template <int NL>
__device__ __forceinline__ float obs_residual(const ChainParams& c, int t, const float (&q)[NL], const float (&v)[NL],
                                              float (&qb)[NL], float (&vb)[NL], bool seed) {
  const float* row = c.obs + (size_t)(t - 1) * c.D;
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    if (c.obs_col[j] >= 0) {
      const float r = __ldg(row + c.obs_col[j]) - q[j];
      acc += r * r;
      if (seed) qb[j] += r * c.inv_so2;
    }
    if (c.obs_col[NL + j] >= 0) {
      const float r = __ldg(row + c.obs_col[NL + j]) - v[j];
      acc += r * r;
      if (seed) vb[j] += r * c.inv_so2;
    }
  }
  return acc;
}

template <int NL>
__device__ __forceinline__ void tape_store(float* __restrict__ tape, size_t slot, size_t U, size_t u,
                                           const float (&q)[NL], const float (&v)[NL]) {
  float* p = tape + slot * (2 * NL) * U + u;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    p[(size_t)j * U] = q[j];
    p[(size_t)(NL + j) * U] = v[j];
  }
}

template <int NL>
__device__ __forceinline__ void tape_load(const float* __restrict__ tape, size_t slot, size_t U, size_t u,
                                          float (&q)[NL], float (&v)[NL]) {
  const float* p = tape + slot * (2 * NL) * U + u;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    q[j] = p[(size_t)j * U];
    v[j] = p[(size_t)(NL + j) * U];
  }
}

// One thread per unit u = w * N + i (window w, particle i): the window's
// forward rollout with its observation and defect terms (Eqs. 2, 4, 5), then
// (grad != 0) the reverse sweep from checkpoints every K steps.
template <int NL, bool FAST>
__device__ __forceinline__ void rollout_unit(const ChainParams& c, const float* __restrict__ X, int N,
                                             const Partials& parts, int grad, int32_t* __restrict__ status,
                                             size_t u) {
  const size_t U = (size_t)N * c.W;
  const int w = (int)(u / N);
  const int i = (int)(u - (size_t)w * N);
  // the window-reduction kernel (next on the stream) ORs in non-finite flags
  if (status && w == 0) status[i] = 0;

  float m[NL], l[NL], b[NL];
  load_params<NL>(c, X, N, i, m, l, b);

  float q[NL], v[NL];
  if (w == 0) {
#pragma unroll
    for (int j = 0; j < NL; ++j) { q[j] = c.s0[j]; v[j] = c.s0[NL + j]; }
  } else {
    const float* xs = X + (size_t)(c.M + (w - 1) * 2 * NL) * N + i;
#pragma unroll
    for (int j = 0; j < NL; ++j) { q[j] = __ldg(xs + (size_t)j * N); v[j] = __ldg(xs + (size_t)(NL + j) * N); }
  }
  const int t0 = (int)(((long long)w * c.T) / c.W);
  const int t1 = (int)(((long long)(w + 1) * c.T) / c.W);
  const int h = t1 - t0;

  float* ckpt = parts.tape;
  float* segbuf = parts.tape + (size_t)c.max_seg * (2 * NL) * U;
  const int K = c.K;

  // ---------------- forward
  float qb[NL], vb[NL];  // unused in the forward pass
  float rss = 0.f;
  for (int k = 0; k < h; ++k) {
    if (grad && (k % K) == 0) tape_store<NL>(ckpt, k / K, U, u, q, v);
    chain_step<NL, FAST>(q, v, m, l, b, c.g, c.dt);
    rss += obs_residual<NL>(c, t0 + k + 1, q, v, qb, vb, false);
  }
  float lp = -0.5f * c.inv_so2 * rss + (float)h * c.obs_const;

  // defect term against the next window's shooting state
  float nb[2 * NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) { qb[j] = 0.f; vb[j] = 0.f; }
  if (w < c.W - 1) {
    const float* xs = X + (size_t)(c.M + w * 2 * NL) * N + i;
    float dss = 0.f;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const float dq = __ldg(xs + (size_t)j * N) - q[j];
      const float dv = __ldg(xs + (size_t)(NL + j) * N) - v[j];
      dss += dq * dq + dv * dv;
      qb[j] = dq * c.inv_sd2;        // d/ds_end of -|d|^2/(2 sd^2)
      vb[j] = dv * c.inv_sd2;
      nb[j] = -dq * c.inv_sd2;       // d/ds^s_{w+1}
      nb[NL + j] = -dv * c.inv_sd2;
    }
    lp += -0.5f * c.inv_sd2 * dss + c.def_const;
  } else {
#pragma unroll
    for (int j = 0; j < 2 * NL; ++j) nb[j] = 0.f;
  }
  parts.lp[(size_t)w * N + i] = lp;
  if (!grad) return;

  // ---------------- reverse sweep
  float mb[NL], lb[NL], bb[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) { mb[j] = 0.f; lb[j] = 0.f; bb[j] = 0.f; }
  float qh[NL], vh[NL];  // state s_{k+1} (output of the step being reversed)
#pragma unroll
  for (int j = 0; j < NL; ++j) { qh[j] = q[j]; vh[j] = v[j]; }
  const int nseg = (h + K - 1) / K;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int a = sg * K;
    const int e = min(a + K, h);
    float qs[NL], vs[NL];
    tape_load<NL>(ckpt, sg, U, u, qs, vs);
    // recompute s_a .. s_{e-1} into the segment buffer
    for (int k = a; k < e; ++k) {
      tape_store<NL>(segbuf, k - a, U, u, qs, vs);
      if (k + 1 < e) chain_step<NL, FAST>(qs, vs, m, l, b, c.g, c.dt);
    }
    for (int k = e - 1; k >= a; --k) {
      // observation at time t0+k+1 depends on s_{k+1}
      obs_residual<NL>(c, t0 + k + 1, qh, vh, qb, vb, true);
      tape_load<NL>(segbuf, k - a, U, u, qs, vs);
      chain_step_vjp<NL, FAST>(qs, vs, m, l, b, c.g, c.dt, qb, vb, mb, lb, bb);
#pragma unroll
      for (int j = 0; j < NL; ++j) { qh[j] = qs[j]; vh[j] = vs[j]; }
    }
  }

  // ---------------- write partial gradients
  float* th = parts.th + (size_t)w * c.M * N + i;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    if (c.mass_theta[j] >= 0) th[(size_t)c.mass_theta[j] * N] = mb[j];
    if (c.length_theta[j] >= 0) th[(size_t)c.length_theta[j] * N] = lb[j];
    if (c.damp_theta[j] >= 0) th[(size_t)c.damp_theta[j] * N] = bb[j];
  }
  float* st = parts.start + (size_t)w * 2 * NL * N + i;
  float* nx = parts.next + (size_t)w * 2 * NL * N + i;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    st[(size_t)j * N] = qb[j];
    st[(size_t)(NL + j) * N] = vb[j];
    nx[(size_t)j * N] = nb[j];
    nx[(size_t)(NL + j) * N] = nb[NL + j];
  }
}

template <int NL, bool FAST>
__global__ void __launch_bounds__(128, PDS_ROLLOUT_MINB) rollout_kernel(const ChainParams c, const float* __restrict__ X,
                                                                        int N, Partials parts, int grad,
                                                                        int32_t* __restrict__ status) {
  const size_t U = (size_t)N * c.W;
  const size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= U) return;
  rollout_unit<NL, FAST>(c, X, N, parts, grad, status, u);
}

// Persistent rollout over several problems with the same chain length
// (batched execution): blocks take work items -- 128 consecutive units of
// one problem -- from a list sorted by decreasing cost (longest windows
// first), through an atomic counter, so problems of uneven size and window
// length share the launch and balance across SMs.  The problem's parameters
// are staged in shared memory for the item.
template <int NL, bool FAST>
__global__ void __launch_bounds__(128, PDS_ROLLOUT_MINB) batch_rollout_kernel(const BatchJob* __restrict__ jobs,
                                                                              const WorkItem* __restrict__ items,
                                                                              int n_items,
                                                                              unsigned int* __restrict__ counter,
                                                                              int grad) {
  __shared__ ChainParams cs;
  __shared__ int item;
  constexpr int kWords = sizeof(ChainParams) / sizeof(int);
  static_assert(sizeof(ChainParams) % sizeof(int) == 0, "ChainParams must be word sized");
  for (;;) {
    if (threadIdx.x == 0) item = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int it = item;
    if (it >= n_items) break;
    const WorkItem wi = items[it];
    const BatchJob* job = jobs + wi.job;
    const int* src = reinterpret_cast<const int*>(&job->c);
    int* dst = reinterpret_cast<int*>(&cs);
    for (int k = threadIdx.x; k < kWords; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    const size_t u = (size_t)wi.unit0 + threadIdx.x;
    const int N = job->N;
    if (u < (size_t)N * cs.W) rollout_unit<NL, FAST>(cs, job->X, N, job->parts, grad, job->status, u);
    __syncthreads();
  }
}

template <int NL>
int batch_rollout_blocks_per_sm_nl(int fast) {
  int nb = 0;
  if (fast)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_rollout_kernel<NL, true>, 128, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_rollout_kernel<NL, false>, 128, 0);
  return nb;
}

template <int NL>
cudaError_t launch_batch_rollout_nl(const BatchJob* jobs, const WorkItem* items, int n_items, unsigned int* counter,
                                    int grad, int fast, int blocks, cudaStream_t st) {
  if (fast)
    batch_rollout_kernel<NL, true><<<blocks, 128, 0, st>>>(jobs, items, n_items, counter, grad);
  else
    batch_rollout_kernel<NL, false><<<blocks, 128, 0, st>>>(jobs, items, n_items, counter, grad);
  return cudaGetLastError();
}

// f_sim for N parameter vectors from s0: states [T+1][S][N].
template <int NL>
__global__ void __launch_bounds__(128) simulate_kernel(const ChainParams c, const float* __restrict__ theta, int N,
                                                       float* __restrict__ states) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  float m[NL], l[NL], b[NL];
  load_params<NL>(c, theta, N, i, m, l, b);
  float q[NL], v[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) { q[j] = c.s0[j]; v[j] = c.s0[NL + j]; }
  const size_t SN = (size_t)2 * NL * N;
  for (int t = 0; t <= c.T; ++t) {
    if (t > 0) chain_step<NL, false>(q, v, m, l, b, c.g, c.dt);
    float* out = states + (size_t)t * SN + i;
#pragma unroll
    for (int j = 0; j < NL; ++j) { out[(size_t)j * N] = q[j]; out[(size_t)(NL + j) * N] = v[j]; }
  }
}

template <int NL>
cudaError_t launch_rollout_nl(const ChainParams& c, const float* X, int N, const Partials& parts, int grad,
                              int32_t* status, cudaStream_t st) {
  const size_t U = (size_t)N * c.W;
  const unsigned blocks = (unsigned)((U + 127) / 128);
  if (c.fast_math)
    rollout_kernel<NL, true><<<blocks, 128, 0, st>>>(c, X, N, parts, grad, status);
  else
    rollout_kernel<NL, false><<<blocks, 128, 0, st>>>(c, X, N, parts, grad, status);
  return cudaGetLastError();
}

template <int NL>
cudaError_t launch_simulate_nl(const ChainParams& c, const float* theta, int N, float* states, cudaStream_t st) {
  simulate_kernel<NL><<<(N + 127) / 128, 128, 0, st>>>(c, theta, N, states);
  return cudaGetLastError();
}

}  // namespace pds
