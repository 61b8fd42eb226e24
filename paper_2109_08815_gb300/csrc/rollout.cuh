// Fused window rollout + hand-written reverse adjoint for planar point-mass
// chains (one thread per particle-window unit).
//
// Forward dynamics (Appendix B-A, Eq. dynamics): the articulated-body
// recursion specialised to a planar chain whose links are massless rods of
// length l_i with a point mass m_i at the tip.  Each link carries a frame
// whose first axis e_i runs along the rod (joint i to mass i) and whose second
// axis p_i is the direction the mass moves when joint i turns; in world
// coordinates e_i = (sin phi_i, -cos phi_i), p_i = (cos phi_i, sin phi_i) with
// phi_i = q_1 + .. + q_i, and the frame of link i+1 is that of link i turned by
// q_{i+1}.  Because a revolute joint carries no moment and the rod is
// massless, the articulated inertia that link i passes to its parent is rank
// one along its own rod: K_i = k_i e_i e_i^T.  With link i+1's axis at
// (c, s) = (cos q_{i+1}, sin q_{i+1}) in link i's frame, the general step
// A_i = K_{i+1} + m_i I, K_i = A_i - A_i p p^T A_i / (p^T A_i p) reduces to
//   h_i = m_i + k_{i+1} s^2,   k_i = m_i (m_i + k_{i+1}) / h_i,
// so the inward pass (i = n..1, k_{n+1} = 0, bias B_{n+1} = 0, tau_{n+1} = 0)
// needs one reciprocal per link:
//   (Be, Bp) = B_{i+1} turned into link i's frame,
//   y_i = k_{i+1} s c,   z_i = m_i + k_{i+1} c^2,   w_i = omega_i^2 l_i,
//   be = Be - w_i z_i - m_i g cos phi_i,   bp = Bp - w_i y_i + m_i g sin phi_i,
//   f_i = ((tau_i - tau_{i+1}) / l_i - bp) / h_i,
//   B_i = (be + f_i y_i, (tau_i - tau_{i+1}) / l_i),
// (B_i is the force link i's parent applies at joint i less K_i a_{i-1}).  The
// outward pass (a_0 = 0) turns the joint acceleration a_{i-1} into link i's
// frame, (ae, ap), and gives the tip acceleration and absolute angular
// acceleration
//   a_i = (ae - w_i, f_i - (y_i / h_i) ae),   alpha_i = (a_i,p - ap) / l_i,
// with qdd_i = alpha_i - alpha_{i-1}.  Semi-implicit Euler then updates
// qd += qdd dt, q += qd dt (the new velocity).  The recursion is the
// textbook one written in link frames; the oracle runs the general spatial
// algorithm, so the two agree only through the dynamics.
//
// The adjoint of one step (Appendix B-A: gradients through f_step by the
// chain rule / adjoint method) differentiates the implicit relation
// ID(q, qd, qdd) = tau instead of the recursion: one solve with the same
// rank-1 articulated inertias gives mu = H^-1 abar, and the gradient of
// mu^T ID for point masses is a closed-form sum over the links (see
// chain_step_vjp).  The reverse step therefore never re-runs the forward
// recursion; it needs only the step's input state and output velocity,
// which the tape holds.
//
// Every fused multiply-add is written out as fmaf and the file is compiled
// with -fmad=false, so the arithmetic is the same in the single-problem and
// the batched kernels whatever the compiler's context: the two give the
// same results bit for bit.
#pragma once

#include "pds_internal.cuh"

// Resident 128-thread blocks per SM the rollout is compiled for: 3 keeps
// chains of up to 5 links in registers; longer chains would spill at 168
// registers and get 2 (255 registers).
#ifdef PDS_ROLLOUT_MINB
#define PDS_ROLLOUT_BLOCKS(NL) (PDS_ROLLOUT_MINB)
#else
#define PDS_ROLLOUT_BLOCKS(NL) ((NL) <= 5 ? 3 : 2)
#endif

namespace pds {

// Lane types.  The step arithmetic is written once for a lane type V: a
// float (one unit per thread) or a float2 holding the same quantity of two
// units side by side, whose arithmetic issues as the paired FP32
// instructions of sm_100 and later (__ffma2_rn, __fmul2_rn, __fadd2_rn).
// Each component of a paired operation rounds exactly as the scalar one, so
// both lane types give the same bits for a unit.
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
// a - b is a + (-b) exactly in IEEE arithmetic
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __fadd2_rn(a, vneg(b)); }
template <class V>
__device__ __forceinline__ V vsplat(float x);
template <>
__device__ __forceinline__ float vsplat<float>(float x) { return x; }
template <>
__device__ __forceinline__ float2 vsplat<float2>(float x) { return make_float2(x, x); }

// sin/cos and reciprocal: CUDA's accurate functions, or (FAST) the hardware
// approximations __sincosf / __fdividef, which the parity tests also cover.
template <bool FAST>
__device__ __forceinline__ void sc(float x, float* s, float* c) {
  if (FAST) __sincosf(x, s, c);
  else sincosf(x, s, c);
}
template <bool FAST>
__device__ __forceinline__ void sc(float2 x, float2* s, float2* c) {
  sc<FAST>(x.x, &s->x, &c->x);
  sc<FAST>(x.y, &s->y, &c->y);
}
template <bool FAST>
__device__ __forceinline__ float rcp(float x) {
  return FAST ? __fdividef(1.0f, x) : 1.0f / x;
}
template <bool FAST>
__device__ __forceinline__ float2 rcp(float2 x) {
  return make_float2(rcp<FAST>(x.x), rcp<FAST>(x.y));
}

// Per-particle link parameters, with the loop-invariant 1 / l and m g.
template <int NL, class V = float>
struct Links {
  V m[NL], l[NL], b[NL];
  V il[NL], mg[NL];
};

// Joint rotations (sin q_i, cos q_i) and absolute-angle (sin, cos) by
// composing them along the chain.
template <int NL, bool FAST, class V>
__device__ __forceinline__ void joint_trig(const V (&q)[NL], V (&sq)[NL], V (&cq)[NL], V (&S)[NL], V (&C)[NL]) {
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    sc<FAST>(q[i], &sq[i], &cq[i]);
    if (i == 0) {
      S[0] = sq[0];
      C[0] = cq[0];
    } else {
      S[i] = vfma(S[i - 1], cq[i], vmul(C[i - 1], sq[i]));
      C[i] = vfma(C[i - 1], cq[i], vmul(vneg(S[i - 1]), sq[i]));
    }
  }
}

// Forward step in place.
template <int NL, bool FAST, class V>
__device__ __forceinline__ void chain_step(V (&q)[NL], V (&v)[NL], const Links<NL, V>& P, float dt_) {
  const V dt = vsplat<V>(dt_);
  const V zero = vsplat<V>(0.f);
  V sq[NL], cq[NL], S[NL], C[NL], o2[NL], w[NL], tau[NL];
  joint_trig<NL, FAST>(q, sq, cq, S, C);
  {
    V om = zero;
#pragma unroll
    for (int i = 0; i < NL; ++i) {
      om = (i == 0) ? v[0] : vadd(om, v[i]);
      o2[i] = vmul(om, om);
      w[i] = vmul(o2[i], P.l[i]);
      tau[i] = vmul(vneg(P.b[i]), v[i]);
    }
  }
  V f[NL], x[NL];
  V Bce = zero, Bcp = zero, kc = zero;
#pragma unroll
  for (int i = NL - 1; i >= 0; --i) {
    const V dtau = (i + 1 < NL) ? vfma(vneg(P.b[i]), v[i], vneg(tau[i + 1])) : tau[i];
    V Be = zero, Bp = zero, h = P.m[i], y = zero, z = P.m[i];
    if (i + 1 < NL) {
      const V s1 = sq[i + 1], c1 = cq[i + 1];
      Be = vfma(Bce, c1, vmul(vneg(Bcp), s1));
      Bp = vfma(Bce, s1, vmul(Bcp, c1));
      const V ks = vmul(kc, s1);
      h = vfma(ks, s1, P.m[i]);
      y = vmul(ks, c1);
      z = vfma(vmul(kc, c1), c1, P.m[i]);
    }
    const V ih = rcp<FAST>(h);
    const V be = vfma(vneg(P.mg[i]), C[i], vfma(vneg(w[i]), z, Be));
    // the outermost link (i = NL - 1) has y = 0, Be = Bp = 0: the terms on
    // those zeros are left out (the same values; no instruction spent on them)
    const V bp = (i + 1 < NL) ? vfma(P.mg[i], S[i], vfma(vneg(w[i]), y, Bp)) : vmul(P.mg[i], S[i]);
    const V ft = vmul(vfma(dtau, P.il[i], vneg(bp)), ih);
    f[i] = ft;
    x[i] = (i + 1 < NL) ? vmul(y, ih) : zero;
    Bce = (i + 1 < NL) ? vfma(ft, y, be) : be;
    Bcp = vmul(dtau, P.il[i]);
    kc = vmul(vmul(P.m[i], (i + 1 < NL) ? vadd(P.m[i], kc) : P.m[i]), ih);
  }
  V Ae = zero, Ap = zero, alp = zero;
#pragma unroll
  for (int i = 0; i < NL; ++i) {
    V ae = zero, ap = zero;
    if (i > 0) {
      ae = vfma(cq[i], Ae, vmul(sq[i], Ap));
      ap = vfma(cq[i], Ap, vmul(vneg(sq[i]), Ae));
    }
    // the base link (i = 0) has ae = ap = 0
    const V An = (i > 0) ? vfma(vneg(x[i]), ae, f[i]) : f[0];
    const V d = (i > 0) ? vsub(An, ap) : An;
    const V al = vmul(d, P.il[i]);
    Ae = vfma(vneg(o2[i]), P.l[i], ae);
    Ap = An;
    // qdd = al - alp with al's product fused: written out, so that every
    // lane type rounds it the same way whatever the compiler contracts
    const V qdd = (i > 0) ? vfma(d, P.il[i], vneg(alp)) : al;
    alp = al;
    v[i] = vfma(qdd, dt, v[i]);
    q[i] = vfma(v[i], dt, q[i]);
  }
}

// Reverse of one step.  On entry (qb, vb) is the adjoint of the step's
// output state (q', v'); on exit it is the adjoint of its input state
// (q, v), and the adjoints of the link parameters are accumulated into
// mb, lb, bb.  v2 = v' is the step's output velocity.
//
// Euler (q' = q + v' dt, v' = v + qdd dt) hands the joint accelerations the
// adjoint abar = (vb + qb dt) dt.  For the dynamics qdd = FD(q, v; m, l, b)
// the reverse uses the inverse-dynamics identity instead of the derivative
// of the articulated-body recursion: FD is the solution of
// ID(q, v, qdd; m, l) + b o v = 0 for the actual qdd, with ID's Jacobian in
// qdd the mass matrix H (symmetric), so
//   abar^T dqdd/dx = -d/dx [ mu^T (ID(q, v, qdd) + b o v) ],  mu = H^-1 abar,
// with mu and qdd held fixed (the adjoint method applied to the implicit
// relation, Appendix B-A).  mu comes from the same rank-1 articulated
// recursion as the forward step with no velocity, gravity or damping terms
// and abar as the joint torques.  For point masses at the link tips,
//   mu^T ID = sum_k m_k (A_k + g y) . delta_k,
//   A_k = sum_{j<=k} l_j (alpha_j p_j - omega_j^2 e_j),   (tip acceleration)
//   delta_k = sum_{j<=k} l_j Lambda_j p_j,                (tip motion under mu)
// with e_j = (sin phi_j, -cos phi_j), p_j = (cos phi_j, sin phi_j), phi,
// omega, alpha and Lambda the partial sums of q, v, qdd and mu over the
// joints up to j.  With the suffix sums F_j = sum_{k>=j} m_k (A_k + g y) and
// D_j = sum_{k>=j} m_k delta_k its gradient is, link by link,
//   d/dm_k   = (A_k + g y) . delta_k
//   d/dl_j   = alpha_j p_j.D_j - omega_j^2 e_j.D_j + Lambda_j p_j.F_j
//   d/domega_j = -2 omega_j l_j e_j.D_j
//   d/dphi_j = l_j (-alpha_j e_j.D_j - omega_j^2 p_j.D_j - Lambda_j e_j.F_j)
// and d/dq_i, d/dv_i are the suffix sums over j >= i of d/dphi_j and
// d/domega_j (plus mu_i b_i for v_i); the damping term gives d/db_i = mu_i v_i.
// qdd is recovered from the taped velocities as (v' - v) / dt: its FP32
// error, half an ulp of v' over dt, stays far below the gradient tolerance.
// LEN = false leaves out d/dl (p_j.F_j and the length adjoint lb), for
// problems with no link length among the parameters; every other output is
// the same bits.
template <int NL, bool FAST, bool LEN = true, class V>
__device__ __forceinline__ void chain_step_vjp(const V (&q)[NL], const V (&v)[NL], const V (&v2)[NL],
                                               const Links<NL, V>& P, float g_, float dt_, float idt_, V (&qb)[NL],
                                               V (&vb)[NL], V (&mb)[NL], V (&lb)[NL], V (&bb)[NL]) {
  const V dt = vsplat<V>(dt_), idt = vsplat<V>(idt_), g = vsplat<V>(g_);
  const V zero = vsplat<V>(0.f);
  // ---- Euler: vb' += qb dt (qb passes through unchanged); abar = vb' dt
#pragma unroll
  for (int i = 0; i < NL; ++i) vb[i] = vfma(qb[i], dt, vb[i]);
  V sq[NL], cq[NL], S[NL], C[NL];
  joint_trig<NL, FAST>(q, sq, cq, S, C);
  // ---- mu = H^-1 abar: inward pass (the articulated inertias k_i) ...
  V f[NL], x[NL];
  {
    V Bce = zero, Bcp = zero, kc = zero;
#pragma unroll
    for (int i = NL - 1; i >= 0; --i) {
      const V dtau = vmul((i + 1 < NL) ? vsub(vb[i], vb[i + 1]) : vb[i], dt);  // abar_i - abar_{i+1}
      V Be = zero, Bp = zero, h = P.m[i], y = zero;
      if (i + 1 < NL) {
        const V s1 = sq[i + 1], c1 = cq[i + 1];
        Be = vfma(Bce, c1, vmul(vneg(Bcp), s1));
        Bp = vfma(Bce, s1, vmul(Bcp, c1));
        const V ks = vmul(kc, s1);
        h = vfma(ks, s1, P.m[i]);
        y = vmul(ks, c1);
      }
      const V ih = rcp<FAST>(h);
      const V ft = vmul(vfma(dtau, P.il[i], vneg(Bp)), ih);
      f[i] = ft;
      x[i] = (i + 1 < NL) ? vmul(y, ih) : zero;
      Bce = (i + 1 < NL) ? vfma(ft, y, Be) : Be;
      Bcp = vmul(dtau, P.il[i]);
      kc = vmul(vmul(P.m[i], (i + 1 < NL) ? vadd(P.m[i], kc) : P.m[i]), ih);
    }
  }
  // ... outward pass (Lambda = absolute angular accelerations of the
  // solution), with the prefix sums A_k + g y and delta_k
  V Lam[NL], mu[NL], om[NL], al[NL], Gx[NL], Gy[NL], dx[NL], dy[NL];
  {
    V Ae = zero, Ap = zero, o = zero, a = zero, Ax = zero, Ay = zero, ddx = zero, ddy = zero;
#pragma unroll
    for (int i = 0; i < NL; ++i) {
      V ae = zero, ap = zero;
      if (i > 0) {
        ae = vfma(cq[i], Ae, vmul(sq[i], Ap));
        ap = vfma(cq[i], Ap, vmul(vneg(sq[i]), Ae));
      }
      const V An = (i > 0) ? vfma(vneg(x[i]), ae, f[i]) : f[0];
      const V d = (i > 0) ? vsub(An, ap) : An;
      Lam[i] = vmul(d, P.il[i]);
      mu[i] = (i > 0) ? vfma(d, P.il[i], vneg(Lam[i - 1])) : Lam[0];  // mu_i = Lambda_i - Lambda_{i-1}, fused
      Ae = ae;
      Ap = An;
      o = (i == 0) ? v[0] : vadd(o, v[i]);
      a = vfma(vsub(v2[i], v[i]), idt, a);
      om[i] = o;
      al[i] = a;
      const V o2 = vmul(o, o);
      const V ux = vfma(a, C[i], vmul(vneg(o2), S[i])), uy = vfma(a, S[i], vmul(o2, C[i]));
      Ax = vfma(P.l[i], ux, Ax);
      Ay = vfma(P.l[i], uy, Ay);
      const V ll = vmul(P.l[i], Lam[i]);
      ddx = vfma(ll, C[i], ddx);
      ddy = vfma(ll, S[i], ddy);
      Gx[i] = Ax;
      Gy[i] = vadd(Ay, g);
      dx[i] = ddx;
      dy[i] = ddy;
    }
  }
  // ---- the gradient of -mu^T (ID + b o v), suffix sums from the tip
  const V m2 = vsplat<V>(-2.f);
  V Fx = zero, Fy = zero, Dx = zero, Dy = zero, sphi = zero, som = zero;
#pragma unroll
  for (int i = NL - 1; i >= 0; --i) {
    const V m = P.m[i];
    Fx = vfma(m, Gx[i], Fx);
    Fy = vfma(m, Gy[i], Fy);
    Dx = vfma(m, dx[i], Dx);
    Dy = vfma(m, dy[i], Dy);
    const V eD = vfma(S[i], Dx, vmul(vneg(C[i]), Dy)), pD = vfma(C[i], Dx, vmul(S[i], Dy));
    const V eF = vfma(S[i], Fx, vmul(vneg(C[i]), Fy));
    const V o2 = vmul(om[i], om[i]);
    mb[i] = vsub(mb[i], vfma(Gx[i], dx[i], vmul(Gy[i], dy[i])));
    if constexpr (LEN) {
      const V pF = vfma(C[i], Fx, vmul(S[i], Fy));
      lb[i] = vsub(lb[i], vfma(al[i], pD, vfma(vneg(o2), eD, vmul(Lam[i], pF))));
    }
    bb[i] = vfma(vneg(mu[i]), v[i], bb[i]);
    som = vfma(vmul(vmul(m2, om[i]), P.l[i]), eD, som);
    sphi = vfma(P.l[i], vfma(vneg(al[i]), eD, vfma(vneg(o2), pD, vmul(vneg(Lam[i]), eF))), sphi);
    qb[i] = vsub(qb[i], sphi);
    vb[i] = vsub(vb[i], vfma(mu[i], P.b[i], som));
  }
}

// Load the physical parameters of particle i (defaults overridden by theta).
template <int NL, bool FAST>
__device__ __forceinline__ void load_params(const ChainParams& c, const float* __restrict__ X, int N, int i,
                                            Links<NL>& P) {
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    P.m[j] = (c.mass_theta[j] >= 0) ? __ldg(X + (size_t)c.mass_theta[j] * N + i) : c.mass[j];
    P.l[j] = (c.length_theta[j] >= 0) ? __ldg(X + (size_t)c.length_theta[j] * N + i) : c.length[j];
    P.b[j] = (c.damp_theta[j] >= 0) ? __ldg(X + (size_t)c.damp_theta[j] * N + i) : c.damping[j];
    P.il[j] = rcp<FAST>(P.l[j]);
    P.mg[j] = P.m[j] * c.g;
  }
}

// Observation residual terms of one step: returns sum of r^2 over observed
// components of state (q, v) at time t (1-based), and if seed != nullptr adds
// d/ds [-r^2 / (2 sigma^2)] = r / sigma^2 to the state adjoint.
//   EVERY (every state component observed): obs is the trajectory's
//     observations in state order, [T][2 NL], read in 8-byte pairs at
//     compile-time offsets with no per-component test;
//   otherwise obs is [T][D] and each component looks up its column.
// The test and the column lookup of the general form, run twice per step,
// cost about 7 % of the chain benchmark's likelihood.
template <int NL, bool EVERY>
__device__ __forceinline__ float obs_residual(const ChainParams& c, const float* __restrict__ obs, int t,
                                              const float (&q)[NL], const float (&v)[NL], float (&qb)[NL],
                                              float (&vb)[NL], bool seed) {
  float acc = 0.f;
  if constexpr (EVERY) {
    const float2* row = reinterpret_cast<const float2*>(obs + (size_t)(t - 1) * (2 * NL));
    auto term = [&](int comp, float o) {  // comp: 0..NL-1 angles, NL..2NL-1 velocities
      if (comp < NL) {
        const float r = o - q[comp];
        acc = fmaf(r, r, acc);
        if (seed) qb[comp] = fmaf(r, c.inv_so2, qb[comp]);
      } else {
        const float r = o - v[comp - NL];
        acc = fmaf(r, r, acc);
        if (seed) vb[comp - NL] = fmaf(r, c.inv_so2, vb[comp - NL]);
      }
    };
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const float2 o = __ldg(row + j);
      term(2 * j, o.x);
      term(2 * j + 1, o.y);
    }
  } else {
    const float* row = obs + (size_t)(t - 1) * c.D;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      if (c.obs_col[j] >= 0) {
        const float r = __ldg(row + c.obs_col[j]) - q[j];
        acc = fmaf(r, r, acc);
        if (seed) qb[j] = fmaf(r, c.inv_so2, qb[j]);
      }
      if (c.obs_col[NL + j] >= 0) {
        const float r = __ldg(row + c.obs_col[NL + j]) - v[j];
        acc = fmaf(r, r, acc);
        if (seed) vb[j] = fmaf(r, c.inv_so2, vb[j]);
      }
    }
  }
  return acc;
}

// The observation seed of one reverse step from a row already loaded (state
// order, pairs): qb, vb += (x_t - s_t) / sigma_obs^2.
template <int NL>
__device__ __forceinline__ void obs_seed_pairs(const ChainParams& c, const float2 (&o)[NL], const float (&q)[NL],
                                               const float (&v)[NL], float (&qb)[NL], float (&vb)[NL]) {
#pragma unroll
  for (int j = 0; j < NL; ++j) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int comp = 2 * j + e;
      const float ov = e ? o[j].y : o[j].x;
      if (comp < NL) qb[comp] = fmaf(ov - q[comp], c.inv_so2, qb[comp]);
      else vb[comp - NL] = fmaf(ov - v[comp - NL], c.inv_so2, vb[comp - NL]);
    }
  }
}

// Asynchronous 8-byte copy global -> shared (cp.async), its group commit,
// and the wait for all but the A newest groups.
__device__ __forceinline__ void cp_async8(float2* dst_smem, const float2* src_global) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src_global)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int A>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(A) : "memory"); }

// The K = 1 reverse sweep prefetches each taped state kRingAhead steps
// before its use into a ring of kRingAhead + 1 shared-memory slots per
// thread.
#ifndef PDS_RING_AHEAD
#define PDS_RING_AHEAD 2
#endif
constexpr int kRingAhead = PDS_RING_AHEAD;
constexpr int kRingSlots = kRingAhead + 1;
// Unroll factor of the single-problem kernel's K = 1 reverse loop.
#ifndef PDS_ROLLOUT_RU
#define PDS_ROLLOUT_RU 2
#endif

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

// The checkpoint tape is thread-contiguous, [slot][U][2 NL]: a unit's state
// (q, v) is 2 NL consecutive floats, moved as NL 8-byte pairs at immediate
// offsets (a warp still covers 32 x 8 NL contiguous bytes per slot).  Pair j
// holds state components 2j and 2j+1 (angles 0..NL-1, then velocities).
template <int NL>
__device__ __forceinline__ float state_comp(const float (&q)[NL], const float (&v)[NL], int comp) {
  return comp < NL ? q[comp] : v[comp - NL];
}
template <int NL>
__device__ __forceinline__ void set_comp(float (&q)[NL], float (&v)[NL], int comp, float x) {
  if (comp < NL) q[comp] = x;
  else v[comp - NL] = x;
}
template <int NL>
__device__ __forceinline__ void ckpt_store(float* __restrict__ tape, size_t slot, size_t U, size_t u,
                                           const float (&q)[NL], const float (&v)[NL]) {
  float2* p = reinterpret_cast<float2*>(tape) + (slot * U + u) * NL;
#pragma unroll
  for (int j = 0; j < NL; ++j) p[j] = make_float2(state_comp<NL>(q, v, 2 * j), state_comp<NL>(q, v, 2 * j + 1));
}
// pairs of one state at p[j * stride] (stride 1: the tape; the block size:
// the shared-memory ring)
template <int NL>
__device__ __forceinline__ void pairs_load(const float2* __restrict__ p, size_t stride, float (&q)[NL],
                                           float (&v)[NL]) {
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    const float2 x = p[(size_t)j * stride];
    set_comp<NL>(q, v, 2 * j, x.x);
    set_comp<NL>(q, v, 2 * j + 1, x.y);
  }
}
template <int NL>
__device__ __forceinline__ void ckpt_load(const float* __restrict__ tape, size_t slot, size_t U, size_t u,
                                          float (&q)[NL], float (&v)[NL]) {
  pairs_load<NL>(reinterpret_cast<const float2*>(tape) + (slot * U + u) * NL, 1, q, v);
}

// One thread per unit u = w * N + i (window w, particle i): the window's
// forward rollout with its observation and defect terms (Eqs. 2, 4, 5), then
// (grad != 0) the reverse sweep from checkpoints every K steps.
// seg (may be NULL): the thread's K slots for the recomputed states of the
// segment being reversed, seg[slot * 2 NL * seg_stride + var * seg_stride]
// -- shared memory when they fit there, else the segment part of the tape.
//
// CS (constrained SVGD, Sec. IV-E): the window's likelihood is the
// observation term only; its defect g_def,w+1 = ||s^s_{w+1} - s_end||^2 /
// sigma_def^2 is a constraint with multiplier lam = X[row M + (W-1) S + w].
// A second adjoint, seeded only at the window's end with
// -dPsi/ds_end = 2 (lam + c g) (s^s_{w+1} - s_end) / sigma_def^2, runs
// through the same recomputed steps: th2 receives its theta part, start the
// sum of both adjoints, next the direct -dPsi/ds^s_{w+1}, gdef the value g.
// RU: unroll factor of the K = 1 reverse loop (2 in the single-problem
// kernel; the batched kernel, which holds both observation forms, runs
// slower unrolled).
template <int NL, bool FAST, bool CS = false, bool EVERY = false, int RU = 1, bool LEN = true>
__device__ __forceinline__ void rollout_unit(const ChainParams& c, const float* __restrict__ X, int N,
                                             const Partials& parts, int grad, int32_t* __restrict__ status,
                                             size_t u, float* seg = nullptr, size_t seg_stride = 0) {
  // unit u = (r W + w) N + i: trajectory r, its window w, particle i
  const size_t U = (size_t)N * c.W * c.R;
  const int wg = (int)(u / N);
  const int i = (int)(u - (size_t)wg * N);
  const int r = wg / c.W, w = wg - r * c.W;
  const float* obs = EVERY ? c.obs_s + (size_t)r * c.T * (2 * NL) : c.obs + (size_t)r * c.T * c.D;
  const int shoot0 = c.M + r * (c.W - 1) * 2 * NL;  // first shooting-state row of trajectory r
  // the window-reduction kernel (next on the stream) ORs in non-finite flags
  if (status && wg == 0) status[i] = 0;

  Links<NL> P;
  load_params<NL, FAST>(c, X, N, i, P);

  float q[NL], v[NL];
  if (w == 0) {
#pragma unroll
    for (int j = 0; j < NL; ++j) { q[j] = c.s0[r * kMaxState + j]; v[j] = c.s0[r * kMaxState + NL + j]; }
  } else {
    const float* xs = X + (size_t)(shoot0 + (w - 1) * 2 * NL) * N + i;
#pragma unroll
    for (int j = 0; j < NL; ++j) { q[j] = __ldg(xs + (size_t)j * N); v[j] = __ldg(xs + (size_t)(NL + j) * N); }
  }
  const int t0 = (int)(((long long)w * c.T) / c.W);
  const int t1 = (int)(((long long)(w + 1) * c.T) / c.W);
  const int h = t1 - t0;

  float* ckpt = parts.tape;
  float* segbuf = seg ? seg : parts.tape + (size_t)c.max_seg * (2 * NL) * U + u;
  const size_t sstride = seg ? seg_stride : U;
  const int K = c.K;

  // ---------------- forward
  float qb[NL], vb[NL];  // unused in the forward pass
  float rss = 0.f;
  int kk = 0, slot = 0;  // step within the checkpoint stride, checkpoint slot (no division per step)
  for (int k = 0; k < h; ++k) {
    if (grad && kk == 0) ckpt_store<NL>(ckpt, slot, U, u, q, v);
    if (++kk == K) {
      kk = 0;
      ++slot;
    }
    chain_step<NL, FAST>(q, v, P, c.dt);
    rss += obs_residual<NL, EVERY>(c, obs, t0 + k + 1, q, v, qb, vb, false);
  }
  float lp = fmaf(-0.5f * c.inv_so2, rss, (float)h * c.obs_const);

  // defect term against the next window's shooting state
  float nb[2 * NL];
  float qb2[NL], vb2[NL];  // CS: adjoint of -Psi_def
#pragma unroll
  for (int j = 0; j < NL; ++j) { qb[j] = 0.f; vb[j] = 0.f; qb2[j] = 0.f; vb2[j] = 0.f; }
  if (w < c.W - 1) {
    const float* xs = X + (size_t)(shoot0 + w * 2 * NL) * N + i;
    float dss = 0.f;
    float dd[2 * NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      dd[j] = __ldg(xs + (size_t)j * N) - q[j];
      dd[NL + j] = __ldg(xs + (size_t)(NL + j) * N) - v[j];
      dss = fmaf(dd[j], dd[j], dss);
      dss = fmaf(dd[NL + j], dd[NL + j], dss);
    }
    if constexpr (CS) {
      const float g = dss * c.inv_sd2;
      const float lam = __ldg(X + (size_t)(c.M + (c.W - 1) * 2 * NL + w) * N + i);
      const float kap2 = 2.f * fmaf(c.c_mdmm, g, lam) * c.inv_sd2;
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        qb2[j] = kap2 * dd[j];  // -dPsi/ds_end
        vb2[j] = kap2 * dd[NL + j];
        nb[j] = -kap2 * dd[j];  // -dPsi/ds^s_{w+1}
        nb[NL + j] = -kap2 * dd[NL + j];
      }
      if (grad) parts.gdef[(size_t)wg * N + i] = g;
    } else {
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        qb[j] = dd[j] * c.inv_sd2;  // d/ds_end of -|d|^2/(2 sd^2)
        vb[j] = dd[NL + j] * c.inv_sd2;
        nb[j] = -dd[j] * c.inv_sd2;  // d/ds^s_{w+1}
        nb[NL + j] = -dd[NL + j] * c.inv_sd2;
      }
      lp += fmaf(-0.5f * c.inv_sd2, dss, c.def_const);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 2 * NL; ++j) nb[j] = 0.f;
    if constexpr (CS) {
      if (grad) parts.gdef[(size_t)wg * N + i] = 0.f;
    }
  }
  parts.lp[(size_t)wg * N + i] = lp;
  if (!grad) return;
  {
    // the defect's gradient in the next shooting state is final here: written
    // now, it holds no registers through the reverse sweep
    float* nx = parts.next + (size_t)wg * 2 * NL * N + i;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      nx[(size_t)j * N] = nb[j];
      nx[(size_t)(NL + j) * N] = nb[NL + j];
    }
  }

  // ---------------- reverse sweep
  const float idt = 1.0f / c.dt;
  float mb[NL], lb[NL], bb[NL];
  float mb2[NL], lb2[NL], bb2[NL];  // CS: theta adjoint of -Psi_def
#pragma unroll
  for (int j = 0; j < NL; ++j) { mb[j] = 0.f; lb[j] = 0.f; bb[j] = 0.f; mb2[j] = 0.f; lb2[j] = 0.f; bb2[j] = 0.f; }
  float qh[NL], vh[NL];  // state s_{k+1} (output of the step being reversed)
#pragma unroll
  for (int j = 0; j < NL; ++j) { qh[j] = q[j]; vh[j] = v[j]; }
  if (K == 1 && seg) {
    // Every pre-step state is on the tape: no recomputation.  Each state is
    // copied into a ring of kRingSlots shared-memory slots kRingAhead steps
    // ahead (cp.async, no registers held), so its load's latency hides
    // behind that many steps' adjoints.  The ring is pair-major,
    // [kRingSlots][NL][block] float2, in the same shared memory (seg is this
    // thread's float of a [..][block] layout, seg_stride the block size).
    constexpr int RS = kRingSlots;
    float2* ring = reinterpret_cast<float2*>(seg - threadIdx.x) + threadIdx.x;
    auto fetch = [&](int k, int rs) {  // state k into ring slot rs = k mod RS
      if (k >= 0) {
        const float2* src = reinterpret_cast<const float2*>(ckpt) + ((size_t)k * U + u) * NL;
        float2* dst = ring + (size_t)rs * NL * sstride;
#pragma unroll
        for (int j = 0; j < NL; ++j) cp_async8(dst + (size_t)j * sstride, src + j);
      }
      cp_async_commit();
    };
    // Every component observed: the observation row of the next step to
    // reverse is loaded one step ahead, into registers
    [[maybe_unused]] float2 onx[NL];
    const float2* orow = reinterpret_cast<const float2*>(obs) + (size_t)t0 * NL;  // row t0 + k + 1 at orow + k NL
    if constexpr (EVERY) {
#pragma unroll
      for (int j = 0; j < NL; ++j) onx[j] = __ldg(orow + (size_t)(h - 1) * NL + j);
    }
    int rs = (h - 1) % RS;  // ring slot of state k, counted down with k
    {
      int r = rs;
#pragma unroll
      for (int a = 1; a <= kRingAhead; ++a) {
        fetch(h - a, r);
        r = r == 0 ? RS - 1 : r - 1;
      }
    }
#pragma unroll RU
    for (int k = h - 1; k >= 0; --k) {
      fetch(k - kRingAhead, rs == RS - 1 ? 0 : rs + 1);  // (k - kRingAhead) mod RS = (k + 1) mod RS
      cp_async_wait<kRingAhead>();  // the group of state k (kRingAhead groups older than the newest)
      float qs[NL], vs[NL];
      pairs_load<NL>(ring + (size_t)rs * NL * sstride, sstride, qs, vs);
      rs = rs == 0 ? RS - 1 : rs - 1;
      if constexpr (EVERY) {
        float2 ocur[NL];
#pragma unroll
        for (int j = 0; j < NL; ++j) ocur[j] = onx[j];
        if (k > 0) {
#pragma unroll
          for (int j = 0; j < NL; ++j) onx[j] = __ldg(orow + (size_t)(k - 1) * NL + j);
        }
        obs_seed_pairs<NL>(c, ocur, qh, vh, qb, vb);
      } else {
        obs_residual<NL, EVERY>(c, obs, t0 + k + 1, qh, vh, qb, vb, true);
      }
      chain_step_vjp<NL, FAST, LEN>(qs, vs, vh, P, c.g, c.dt, idt, qb, vb, mb, lb, bb);
      if constexpr (CS) chain_step_vjp<NL, FAST, LEN>(qs, vs, vh, P, c.g, c.dt, idt, qb2, vb2, mb2, lb2, bb2);
#pragma unroll
      for (int j = 0; j < NL; ++j) { qh[j] = qs[j]; vh[j] = vs[j]; }
    }
  } else if (K == 1) {
    // Every pre-step state is on the tape: no recomputation.  The state of
    // step k-1 is loaded while step k is reversed, so the load's latency
    // hides behind the step's adjoint.
    float qs[NL], vs[NL], qn[NL] = {}, vn[NL] = {};
    ckpt_load<NL>(ckpt, h - 1, U, u, qs, vs);
    for (int k = h - 1; k >= 0; --k) {
      if (k > 0) ckpt_load<NL>(ckpt, k - 1, U, u, qn, vn);
      obs_residual<NL, EVERY>(c, obs, t0 + k + 1, qh, vh, qb, vb, true);
      chain_step_vjp<NL, FAST, LEN>(qs, vs, vh, P, c.g, c.dt, idt, qb, vb, mb, lb, bb);
      if constexpr (CS) chain_step_vjp<NL, FAST, LEN>(qs, vs, vh, P, c.g, c.dt, idt, qb2, vb2, mb2, lb2, bb2);
#pragma unroll
      for (int j = 0; j < NL; ++j) { qh[j] = qs[j]; vh[j] = vs[j]; qs[j] = qn[j]; vs[j] = vn[j]; }
    }
  }
  const int nseg = K == 1 ? 0 : (h + K - 1) / K;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int a = sg * K;
    const int e = min(a + K, h);
    float qs[NL], vs[NL];
    ckpt_load<NL>(ckpt, sg, U, u, qs, vs);
    // recompute s_a .. s_{e-1} into the segment buffer
    for (int k = a; k < e; ++k) {
      tape_store<NL>(segbuf, k - a, sstride, 0, qs, vs);
      if (k + 1 < e) chain_step<NL, FAST>(qs, vs, P, c.dt);
    }
    for (int k = e - 1; k >= a; --k) {
      // observation at time t0+k+1 depends on s_{k+1}
      obs_residual<NL, EVERY>(c, obs, t0 + k + 1, qh, vh, qb, vb, true);
      tape_load<NL>(segbuf, k - a, sstride, 0, qs, vs);
      chain_step_vjp<NL, FAST, LEN>(qs, vs, vh, P, c.g, c.dt, idt, qb, vb, mb, lb, bb);
      if constexpr (CS) chain_step_vjp<NL, FAST, LEN>(qs, vs, vh, P, c.g, c.dt, idt, qb2, vb2, mb2, lb2, bb2);
#pragma unroll
      for (int j = 0; j < NL; ++j) { qh[j] = qs[j]; vh[j] = vs[j]; }
    }
  }

  // ---------------- write partial gradients
  float* th = parts.th + (size_t)wg * c.M * N + i;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    if (c.mass_theta[j] >= 0) th[(size_t)c.mass_theta[j] * N] = mb[j];
    if (c.length_theta[j] >= 0) th[(size_t)c.length_theta[j] * N] = lb[j];
    if (c.damp_theta[j] >= 0) th[(size_t)c.damp_theta[j] * N] = bb[j];
  }
  if constexpr (CS) {
    float* th2 = parts.th2 + (size_t)wg * c.M * N + i;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      if (c.mass_theta[j] >= 0) th2[(size_t)c.mass_theta[j] * N] = mb2[j];
      if (c.length_theta[j] >= 0) th2[(size_t)c.length_theta[j] * N] = lb2[j];
      if (c.damp_theta[j] >= 0) th2[(size_t)c.damp_theta[j] * N] = bb2[j];
    }
#pragma unroll
    for (int j = 0; j < NL; ++j) { qb[j] += qb2[j]; vb[j] += vb2[j]; }
  }
  float* st = parts.start + (size_t)wg * 2 * NL * N + i;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    st[(size_t)j * N] = qb[j];
    st[(size_t)(NL + j) * N] = vb[j];
  }
}

// Two units per thread: particles i and i + 1 (i even) of one window and
// trajectory, every quantity held as a float2 (particle i in .x, i + 1 in
// .y), so that each FP32 operation of both units' steps issues as one paired
// instruction and the issue slots it frees go to the loads, MUFU and integer
// work.  The arithmetic of each unit is that of rollout_unit operation for
// operation, so the results are the same bits.  Taken for K = 1 (every
// pre-step state on the tape, read back through the shared-memory ring)
// when every state component is observed, with one adjoint (no constrained
// SVGD) and an even particle count.
//   tape: [slot][U / 2][NL] float4, float4 j = components 2j and 2j + 1 of
//         both units (same bytes per slot as the one-unit layout);
//   ring: [kRingSlots][NL][rstride] float4 in shared memory, this thread's
//         column at ring[0];
//   c.obs_b: each observation twice, [R][T][2 NL] float2 = (x, x), read as
//         NL float4 per row.
__device__ __forceinline__ void cp_async16(float4* dst_smem, const float4* src_global) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src_global)
               : "memory");
}

template <int NL>
__device__ __forceinline__ float2 pair_comp(const float2 (&q)[NL], const float2 (&v)[NL], int comp) {
  return comp < NL ? q[comp] : v[comp - NL];
}

template <int NL, bool FAST, bool LEN = true>
__device__ __forceinline__ void rollout_pair_unit(const ChainParams& c, const float* __restrict__ X, int N,
                                                  const Partials& parts, int32_t* __restrict__ status, size_t u,
                                                  float4* ring, int rstride) {
  using V = float2;
  const size_t U = (size_t)N * c.W * c.R;
  const size_t TS = U / 2 * NL;  // float4 per tape slot
  const int wg = (int)(u / N);
  const int i = (int)(u - (size_t)wg * N);
  const int r = wg / c.W, w = wg - r * c.W;
  const float4* obs4 = reinterpret_cast<const float4*>(c.obs_b) + (size_t)r * c.T * NL;  // row t at (t - 1) NL
  const int shoot0 = c.M + r * (c.W - 1) * 2 * NL;
  if (status && wg == 0) *reinterpret_cast<int2*>(status + i) = make_int2(0, 0);
  auto ld2 = [&](const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); };

  Links<NL, V> P;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    P.m[j] = (c.mass_theta[j] >= 0) ? ld2(X + (size_t)c.mass_theta[j] * N + i) : vsplat<V>(c.mass[j]);
    P.l[j] = (c.length_theta[j] >= 0) ? ld2(X + (size_t)c.length_theta[j] * N + i) : vsplat<V>(c.length[j]);
    P.b[j] = (c.damp_theta[j] >= 0) ? ld2(X + (size_t)c.damp_theta[j] * N + i) : vsplat<V>(c.damping[j]);
    P.il[j] = rcp<FAST>(P.l[j]);
    P.mg[j] = vmul(P.m[j], vsplat<V>(c.g));
  }
  V q[NL], v[NL];
  if (w == 0) {
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      q[j] = vsplat<V>(c.s0[r * kMaxState + j]);
      v[j] = vsplat<V>(c.s0[r * kMaxState + NL + j]);
    }
  } else {
    const float* xs = X + (size_t)(shoot0 + (w - 1) * 2 * NL) * N + i;
#pragma unroll
    for (int j = 0; j < NL; ++j) { q[j] = ld2(xs + (size_t)j * N); v[j] = ld2(xs + (size_t)(NL + j) * N); }
  }
  const int t0 = (int)(((long long)w * c.T) / c.W);
  const int t1 = (int)(((long long)(w + 1) * c.T) / c.W);
  const int h = t1 - t0;
  float4* tape = reinterpret_cast<float4*>(parts.tape) + u / 2 * NL;

  // ---------------- forward
  V rss = vsplat<V>(0.f);
  const float4* orow = obs4 + (size_t)t0 * NL;  // row t0 + k + 1
  for (int k = 0; k < h; ++k, orow += NL) {
    float4* tp = tape + (size_t)k * TS;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const V a = pair_comp<NL>(q, v, 2 * j), b = pair_comp<NL>(q, v, 2 * j + 1);
      tp[j] = make_float4(a.x, a.y, b.x, b.y);
    }
    chain_step<NL, FAST>(q, v, P, c.dt);
    V acc = vsplat<V>(0.f);
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      const float4 o = __ldg(orow + j);
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const V ov = e ? make_float2(o.z, o.w) : make_float2(o.x, o.y);
        const V rr = vsub(ov, pair_comp<NL>(q, v, 2 * j + e));
        acc = vfma(rr, rr, acc);
      }
    }
    rss = vadd(rss, acc);
  }
  V lp = vfma(vsplat<V>(-0.5f * c.inv_so2), rss, vsplat<V>((float)h * c.obs_const));

  // defect term against the next window's shooting state
  V nb[2 * NL], qb[NL], vb[NL];
  const V isd2 = vsplat<V>(c.inv_sd2);
#pragma unroll
  for (int j = 0; j < NL; ++j) { qb[j] = vsplat<V>(0.f); vb[j] = vsplat<V>(0.f); }
  if (w < c.W - 1) {
    const float* xs = X + (size_t)(shoot0 + w * 2 * NL) * N + i;
    V dss = vsplat<V>(0.f);
    V dd[2 * NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      dd[j] = vsub(ld2(xs + (size_t)j * N), q[j]);
      dd[NL + j] = vsub(ld2(xs + (size_t)(NL + j) * N), v[j]);
      dss = vfma(dd[j], dd[j], dss);
      dss = vfma(dd[NL + j], dd[NL + j], dss);
    }
#pragma unroll
    for (int j = 0; j < NL; ++j) {
      qb[j] = vmul(dd[j], isd2);
      vb[j] = vmul(dd[NL + j], isd2);
      nb[j] = vmul(vneg(dd[j]), isd2);
      nb[NL + j] = vmul(vneg(dd[NL + j]), isd2);
    }
    lp = vadd(lp, vfma(vsplat<V>(-0.5f * c.inv_sd2), dss, vsplat<V>(c.def_const)));
  } else {
#pragma unroll
    for (int j = 0; j < 2 * NL; ++j) nb[j] = vsplat<V>(0.f);
  }
  *reinterpret_cast<float2*>(parts.lp + (size_t)wg * N + i) = lp;
  {
    float* nx = parts.next + (size_t)wg * 2 * NL * N + i;
#pragma unroll
    for (int j = 0; j < 2 * NL; ++j) *reinterpret_cast<float2*>(nx + (size_t)j * N) = nb[j];
  }

  // ---------------- reverse sweep: state k from the ring, kRingAhead steps ahead
  const float idt = 1.0f / c.dt;
  const V iso2 = vsplat<V>(c.inv_so2);
  V mb[NL], lb[NL], bb[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) { mb[j] = vsplat<V>(0.f); lb[j] = vsplat<V>(0.f); bb[j] = vsplat<V>(0.f); }
  V qh[NL], vh[NL];  // state s_{k+1}
#pragma unroll
  for (int j = 0; j < NL; ++j) { qh[j] = q[j]; vh[j] = v[j]; }
  constexpr int RS = kRingSlots;
  auto fetch = [&](int k, int rs) {
    if (k >= 0) {
      const float4* src = tape + (size_t)k * TS;
      float4* dst = ring + (size_t)rs * NL * rstride;
#pragma unroll
      for (int j = 0; j < NL; ++j) cp_async16(dst + (size_t)j * rstride, src + j);
    }
    cp_async_commit();
  };
  const float4* orev = obs4 + (size_t)t0 * NL;  // row t0 + k + 1 at orev + k NL
  float4 onx[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) onx[j] = __ldg(orev + (size_t)(h - 1) * NL + j);
  int rs = (h - 1) % RS;
  {
    int r2 = rs;
#pragma unroll
    for (int a = 1; a <= kRingAhead; ++a) {
      fetch(h - a, r2);
      r2 = r2 == 0 ? RS - 1 : r2 - 1;
    }
  }
#pragma unroll 1
  for (int k = h - 1; k >= 0; --k) {
    fetch(k - kRingAhead, rs == RS - 1 ? 0 : rs + 1);
    cp_async_wait<kRingAhead>();
    V qs[NL], vs[NL];
    {
      const float4* sl = ring + (size_t)rs * NL * rstride;
#pragma unroll
      for (int j = 0; j < NL; ++j) {
        const float4 x = sl[(size_t)j * rstride];
        const V a = make_float2(x.x, x.y), b = make_float2(x.z, x.w);
        if (2 * j < NL) qs[2 * j] = a; else vs[2 * j - NL] = a;
        if (2 * j + 1 < NL) qs[2 * j + 1] = b; else vs[2 * j + 1 - NL] = b;
      }
    }
    rs = rs == 0 ? RS - 1 : rs - 1;
    float4 ocur[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) ocur[j] = onx[j];
    if (k > 0) {
#pragma unroll
      for (int j = 0; j < NL; ++j) onx[j] = __ldg(orev + (size_t)(k - 1) * NL + j);
    }
#pragma unroll
    for (int j = 0; j < NL; ++j) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int comp = 2 * j + e;
        const V ov = e ? make_float2(ocur[j].z, ocur[j].w) : make_float2(ocur[j].x, ocur[j].y);
        if (comp < NL) qb[comp] = vfma(vsub(ov, qh[comp]), iso2, qb[comp]);
        else vb[comp - NL] = vfma(vsub(ov, vh[comp - NL]), iso2, vb[comp - NL]);
      }
    }
    chain_step_vjp<NL, FAST, LEN>(qs, vs, vh, P, c.g, c.dt, idt, qb, vb, mb, lb, bb);
#pragma unroll
    for (int j = 0; j < NL; ++j) { qh[j] = qs[j]; vh[j] = vs[j]; }
  }

  // ---------------- write partial gradients
  auto st2 = [&](float* p, V x) { *reinterpret_cast<float2*>(p) = x; };
  float* th = parts.th + (size_t)wg * c.M * N + i;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    if (c.mass_theta[j] >= 0) st2(th + (size_t)c.mass_theta[j] * N, mb[j]);
    if (c.length_theta[j] >= 0) st2(th + (size_t)c.length_theta[j] * N, lb[j]);
    if (c.damp_theta[j] >= 0) st2(th + (size_t)c.damp_theta[j] * N, bb[j]);
  }
  float* st = parts.start + (size_t)wg * 2 * NL * N + i;
#pragma unroll
  for (int j = 0; j < NL; ++j) {
    st2(st + (size_t)j * N, qb[j]);
    st2(st + (size_t)(NL + j) * N, vb[j]);
  }
}

// Units [u0, u1) (both even), two per thread.
template <int NL, bool FAST, bool LEN = true>
__global__ void __launch_bounds__(128, 2) rollout_pair_kernel(const ChainParams c,
                                                                          const float* __restrict__ X, int N,
                                                                          Partials parts,
                                                                          int32_t* __restrict__ status, size_t u0,
                                                                          size_t u1) {
  extern __shared__ float4 ring4_sh[];
  const size_t u = u0 + 2 * ((size_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (u >= u1) return;
  rollout_pair_unit<NL, FAST, LEN>(c, X, N, parts, status, u, ring4_sh + threadIdx.x, blockDim.x);
}

// seg_smem: the reverse sweep's recomputed segment states live in dynamic
// shared memory (K x 2 NL x blockDim floats), else in the tape.  EVERY:
// the problem observes every state component.
// Units [u0, u1) of the launch (all N W R units, or those of a group of
// windows whose particle rows have arrived).
template <int NL, bool FAST, bool EVERY, bool LEN = true>
__global__ void __launch_bounds__(128, PDS_ROLLOUT_BLOCKS(NL)) rollout_kernel(const ChainParams c, const float* __restrict__ X,
                                                                        int N, Partials parts, int grad,
                                                                        int32_t* __restrict__ status, int seg_smem,
                                                                        size_t u0, size_t u1) {
  extern __shared__ float seg_sh[];
  const size_t u = u0 + (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= u1) return;
  if (seg_smem)
    rollout_unit<NL, FAST, false, EVERY, PDS_ROLLOUT_RU, LEN>(c, X, N, parts, grad, status, u,
                                                               seg_sh + threadIdx.x, blockDim.x);
  else
    rollout_unit<NL, FAST, false, EVERY, PDS_ROLLOUT_RU, LEN>(c, X, N, parts, grad, status, u);
}

// log p alone (no gradient): the forward sweep needs far fewer registers
// than the reverse, so it runs with more resident blocks.
#ifndef PDS_FWD_BLOCKS
#define PDS_FWD_BLOCKS 5
#endif
template <int NL, bool FAST, bool EVERY>
__global__ void __launch_bounds__(128, PDS_FWD_BLOCKS) rollout_fwd_kernel(const ChainParams c,
                                                                        const float* __restrict__ X, int N,
                                                                        Partials parts, int32_t* __restrict__ status) {
  const size_t U = (size_t)N * c.W * c.R;
  const size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= U) return;
  rollout_unit<NL, FAST, false, EVERY>(c, X, N, parts, 0, status, u);
}

// Constrained-SVGD variant of rollout_kernel (two adjoints per unit).
template <int NL, bool FAST, bool EVERY, bool LEN = true>
__global__ void __launch_bounds__(128, 2) rollout_cs_kernel(const ChainParams c,
                                                                           const float* __restrict__ X, int N,
                                                                           Partials parts, int grad,
                                                                           int32_t* __restrict__ status, int seg_smem) {
  extern __shared__ float seg_sh[];
  const size_t U = (size_t)N * c.W * c.R;
  const size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= U) return;
  if (seg_smem)
    rollout_unit<NL, FAST, true, EVERY, 1, LEN>(c, X, N, parts, grad, status, u, seg_sh + threadIdx.x, blockDim.x);
  else
    rollout_unit<NL, FAST, true, EVERY, 1, LEN>(c, X, N, parts, grad, status, u);
}

// Persistent rollout over several problems with the same chain length
// (batched execution): blocks take work items -- 128 consecutive units of
// one problem -- from a list sorted by decreasing cost (longest windows
// first), through an atomic counter, so problems of uneven size and window
// length share the launch and balance across SMs.  The problem's parameters
// are staged in shared memory for the item.
template <int NL, bool FAST>
__global__ void __launch_bounds__(128, PDS_ROLLOUT_BLOCKS(NL)) batch_rollout_kernel(const BatchJob* __restrict__ jobs,
                                                                              const WorkItem* __restrict__ items,
                                                                              int n_items,
                                                                              unsigned int* __restrict__ counter,
                                                                              int grad, int ring) {
  // ring: dynamic shared memory holds the K = 1 prefetch ring (kRingSlots states per thread)
  extern __shared__ float ring_sh[];
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
    float* seg = (ring && cs.K == 1) ? ring_sh + threadIdx.x : nullptr;
    // a problem that observes every state component takes the residual
    // form without per-component tests, as its single-problem launch does
    constexpr unsigned int kAll = (1u << (2 * NL)) - 1u;
    if (u < (size_t)N * cs.W) {
      if ((cs.obs_mask & kAll) == kAll)
        rollout_unit<NL, FAST, false, true>(cs, job->X, N, job->parts, grad, job->status, u, seg, blockDim.x);
      else
        rollout_unit<NL, FAST, false, false>(cs, job->X, N, job->parts, grad, job->status, u, seg, blockDim.x);
    }
    __syncthreads();
  }
}

// The persistent batched launch with two units per thread (the two-unit
// step of rollout_pair_unit): a work item is 256 consecutive units of one
// problem, whose particle count is even, every state component observed,
// K = 1.  The batch sets it up only for groups whose problems all qualify.
template <int NL, bool FAST>
__global__ void __launch_bounds__(128, 2) batch_rollout_pair_kernel(const BatchJob* __restrict__ jobs,
                                                                   const WorkItem* __restrict__ items, int n_items,
                                                                   unsigned int* __restrict__ counter) {
  extern __shared__ float4 pring_sh[];
  __shared__ ChainParams cs;
  __shared__ int item;
  constexpr int kWords = sizeof(ChainParams) / sizeof(int);
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
    const size_t u = (size_t)wi.unit0 + 2 * (size_t)threadIdx.x;
    const int N = job->N;
    if (u < (size_t)N * cs.W * cs.R)
      rollout_pair_unit<NL, FAST>(cs, job->X, N, job->parts, job->status, u, pring_sh + threadIdx.x, blockDim.x);
    __syncthreads();
  }
}

template <int NL>
int batch_rollout_blocks_per_sm_nl(int fast, int upt) {
  int nb = 0;
  const size_t psmem = (size_t)kRingSlots * NL * 128 * sizeof(float4);
  if (upt == 2) {
    if (fast)
      cudaFuncSetAttribute(batch_rollout_pair_kernel<NL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    else
      cudaFuncSetAttribute(batch_rollout_pair_kernel<NL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
  }
  if (upt == 2 && fast)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_rollout_pair_kernel<NL, true>, 128, psmem);
  else if (upt == 2)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_rollout_pair_kernel<NL, false>, 128, psmem);
  else if (fast)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_rollout_kernel<NL, true>, 128, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_rollout_kernel<NL, false>, 128, 0);
  return nb;
}

template <int NL>
cudaError_t launch_batch_rollout_nl(const BatchJob* jobs, const WorkItem* items, int n_items, unsigned int* counter,
                                    int grad, int fast, int blocks, int ring, int upt, cudaStream_t st) {
  if (upt == 2) {
    if (!grad || !ring) return cudaErrorInvalidValue;
    const size_t psmem = (size_t)kRingSlots * NL * 128 * sizeof(float4);
    // with the staged ChainParams the block can pass 48 KB: opt in (per device)
    const cudaError_t e =
        fast ? cudaFuncSetAttribute(batch_rollout_pair_kernel<NL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)psmem)
             : cudaFuncSetAttribute(batch_rollout_pair_kernel<NL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)psmem);
    if (e != cudaSuccess) return e;
    if (fast)
      batch_rollout_pair_kernel<NL, true><<<blocks, 128, psmem, st>>>(jobs, items, n_items, counter);
    else
      batch_rollout_pair_kernel<NL, false><<<blocks, 128, psmem, st>>>(jobs, items, n_items, counter);
    return cudaGetLastError();
  }
  const size_t smem = ring ? (size_t)kRingSlots * 2 * NL * 128 * sizeof(float) : 0;
  if (fast)
    batch_rollout_kernel<NL, true><<<blocks, 128, smem, st>>>(jobs, items, n_items, counter, grad, ring);
  else
    batch_rollout_kernel<NL, false><<<blocks, 128, smem, st>>>(jobs, items, n_items, counter, grad, ring);
  return cudaGetLastError();
}

// f_sim for N parameter vectors from s0: states [T+1][S][N].
template <int NL>
__global__ void __launch_bounds__(128) simulate_kernel(const ChainParams c, const float* __restrict__ theta, int N,
                                                       float* __restrict__ states) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  Links<NL> P;
  load_params<NL, false>(c, theta, N, i, P);
  float q[NL], v[NL];
#pragma unroll
  for (int j = 0; j < NL; ++j) { q[j] = c.s0[j]; v[j] = c.s0[NL + j]; }
  const size_t SN = (size_t)2 * NL * N;
  for (int t = 0; t <= c.T; ++t) {
    if (t > 0) chain_step<NL, false>(q, v, P, c.dt);
    float* out = states + (size_t)t * SN + i;
#pragma unroll
    for (int j = 0; j < NL; ++j) { out[(size_t)j * N] = q[j]; out[(size_t)(NL + j) * N] = v[j]; }
  }
}

// The two-units-per-thread kernel can take a gradient launch with K = 1,
// every state component observed, one adjoint, an even particle count and an
// even unit range, when its ring fits in 48 KB of shared memory.  It then
// runs when c.units_per_thread asks for it (2), or by default (0) for the
// chain lengths where it measured faster on GB300 (2, 4 and 5 links: its 254
// registers leave 8 warps per SM, against 12 for the one-unit kernel, and
// longer chains spill).
template <int NL>
bool pair_path_applies(const ChainParams& c, int N, size_t u0, size_t nu) {
  constexpr unsigned int kAll = (1u << (2 * NL)) - 1u;
  const bool can = c.K == 1 && !c.csvgd && (c.obs_mask & kAll) == kAll && c.obs_b != nullptr && N % 2 == 0 &&
                   u0 % 2 == 0 && nu % 2 == 0 && (size_t)kRingSlots * NL * 128 * sizeof(float4) <= 48 * 1024;
  if (!can || c.units_per_thread == 1) return false;
  return c.units_per_thread == 2 || NL == 2 || NL == 4 || NL == 5;
}

// nu = 0: all units; otherwise units [u0, u0 + nu) of the gradient kernel.
template <int NL>
cudaError_t launch_rollout_nl(const ChainParams& c, const float* X, int N, const Partials& parts, int grad,
                              int32_t* status, cudaStream_t st, size_t u0, size_t nu) {
  const size_t U = (size_t)N * c.W * c.R;
  if (nu == 0) {
    u0 = 0;
    nu = U;
  } else if (!grad || c.csvgd || u0 + nu > U) {
    return cudaErrorInvalidValue;
  }
  const unsigned blocks = (unsigned)((nu + 127) / 128);
  const size_t u1 = u0 + nu;
  // the reverse sweep's K recomputed states (K = 1: the ring of kRingSlots
  // prefetched states) in shared memory when they fit in the default 48 KB of
  // a block
  const size_t seg_bytes = (size_t)(c.K == 1 ? kRingSlots : c.K) * 2 * NL * 128 * sizeof(float);
  const int seg_smem = (grad && seg_bytes <= 48 * 1024) ? 1 : 0;
  const size_t smem = seg_smem ? seg_bytes : 0;
  constexpr unsigned int kAll = (1u << (2 * NL)) - 1u;
  const bool every = (c.obs_mask & kAll) == kAll;
  // no link length among the parameters: the adjoint step leaves out the
  // length adjoint (the same bits for everything else)
  bool lengths = false;
#pragma unroll
  for (int j = 0; j < NL; ++j) lengths |= c.length_theta[j] >= 0;
  if (c.csvgd) {
    if (c.fast_math && every && !lengths)
      rollout_cs_kernel<NL, true, true, false><<<blocks, 128, smem, st>>>(c, X, N, parts, grad, status, seg_smem);
    else if (c.fast_math && every)
      rollout_cs_kernel<NL, true, true><<<blocks, 128, smem, st>>>(c, X, N, parts, grad, status, seg_smem);
    else if (c.fast_math)
      rollout_cs_kernel<NL, true, false><<<blocks, 128, smem, st>>>(c, X, N, parts, grad, status, seg_smem);
    else
      rollout_cs_kernel<NL, false, false><<<blocks, 128, smem, st>>>(c, X, N, parts, grad, status, seg_smem);
  } else if (!grad) {
    if (c.fast_math && every)
      rollout_fwd_kernel<NL, true, true><<<blocks, 128, 0, st>>>(c, X, N, parts, status);
    else if (c.fast_math)
      rollout_fwd_kernel<NL, true, false><<<blocks, 128, 0, st>>>(c, X, N, parts, status);
    else if (every)
      rollout_fwd_kernel<NL, false, true><<<blocks, 128, 0, st>>>(c, X, N, parts, status);
    else
      rollout_fwd_kernel<NL, false, false><<<blocks, 128, 0, st>>>(c, X, N, parts, status);
  } else if (pair_path_applies<NL>(c, N, u0, nu)) {
    const size_t rsmem = (size_t)kRingSlots * NL * 128 * sizeof(float4);
    const unsigned pblocks = (unsigned)((nu / 2 + 127) / 128);
    if (c.fast_math && !lengths)
      rollout_pair_kernel<NL, true, false><<<pblocks, 128, rsmem, st>>>(c, X, N, parts, status, u0, u1);
    else if (c.fast_math)
      rollout_pair_kernel<NL, true><<<pblocks, 128, rsmem, st>>>(c, X, N, parts, status, u0, u1);
    else
      rollout_pair_kernel<NL, false><<<pblocks, 128, rsmem, st>>>(c, X, N, parts, status, u0, u1);
  } else {
    // the same residual form as the batched kernel takes for the problem
    if (c.fast_math && every && !lengths)
      rollout_kernel<NL, true, true, false><<<blocks, 128, smem, st>>>(c, X, N, parts, grad, status, seg_smem, u0, u1);
    else if (c.fast_math && !lengths)
      rollout_kernel<NL, true, false, false><<<blocks, 128, smem, st>>>(c, X, N, parts, grad, status, seg_smem, u0, u1);
    else if (c.fast_math && every)
      rollout_kernel<NL, true, true><<<blocks, 128, smem, st>>>(c, X, N, parts, grad, status, seg_smem, u0, u1);
    else if (c.fast_math)
      rollout_kernel<NL, true, false><<<blocks, 128, smem, st>>>(c, X, N, parts, grad, status, seg_smem, u0, u1);
    else if (every)
      rollout_kernel<NL, false, true><<<blocks, 128, smem, st>>>(c, X, N, parts, grad, status, seg_smem, u0, u1);
    else
      rollout_kernel<NL, false, false><<<blocks, 128, smem, st>>>(c, X, N, parts, grad, status, seg_smem, u0, u1);
  }
  return cudaGetLastError();
}

template <int NL>
cudaError_t launch_simulate_nl(const ChainParams& c, const float* theta, int N, float* states, cudaStream_t st) {
  simulate_kernel<NL><<<(N + 127) / 128, 128, 0, st>>>(c, theta, N, states);
  return cudaGetLastError();
}

}  // namespace pds
