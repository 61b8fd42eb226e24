"""Operation-counting transcription of the rollout's per-step arithmetic.

Test infrastructure: an independent count of the floating-point operations
that one forward step and one reverse step of the planar point-mass chain
execute on the GPU, to check the roofline numerator that bench.py uses.  The
steps below follow csrc/rollout.cuh's chain_step, obs_residual,
chain_step_vjp and the observation seed operation for operation, on a scalar
type that carries an FP64 value and counts what it executes:

    add, subtract, multiply: 1 flop;  fused multiply-add: 2;
    negation: 0 (an operand modifier on the GPU);
    sin/cos and reciprocal: 0 (they run on the MUFU, not the FMA pipes);
    an operation with a structural zero (a value that is 0 by construction,
    such as the empty accumulators at the chain's ends, known when the
    kernel is compiled): 0 for a product, and a sum or a fused
    multiply-add passes its other term through (an FMA onto a structural
    zero is one product).

Because the values are real FP64 numbers, the same transcription is checked
against the FP64 oracle's dynamics and against finite differences of it
(tests/test_flopcount.py): the operations counted are those of an algorithm
that computes the right step and the right adjoint.  Nothing here is used by
the library.
"""
from __future__ import annotations

import math


class Counter:
    def __init__(self):
        self.flops = 0


class S:
    """A scalar: FP64 value, the counter its operations charge, and whether
    it is a structural zero."""

    __slots__ = ("v", "c", "z")

    def __init__(self, v, c, z=False):
        self.v = float(v)
        self.c = c
        self.z = z

    def _w(self, x):
        return x if isinstance(x, S) else S(x, self.c)

    def __add__(self, o):
        o = self._w(o)
        if self.z or o.z:
            return S(self.v + o.v, self.c, self.z and o.z)
        self.c.flops += 1
        return S(self.v + o.v, self.c)

    def __sub__(self, o):
        o = self._w(o)
        if self.z or o.z:
            return S(self.v - o.v, self.c, self.z and o.z)
        self.c.flops += 1
        return S(self.v - o.v, self.c)

    def __mul__(self, o):
        o = self._w(o)
        if self.z or o.z:
            return S(0.0, self.c, True)
        self.c.flops += 1
        return S(self.v * o.v, self.c)

    def __neg__(self):
        return S(-self.v, self.c, self.z)


def zero(c):
    return S(0.0, c, True)


def fma(a, b, c):
    if a.z or b.z:
        return c
    if c.z:
        return a * b
    a.c.flops += 2
    return S(a.v * b.v + c.v, a.c)


def sincos(x):
    return S(math.sin(x.v), x.c), S(math.cos(x.v), x.c)


def rcp(x):
    return S(1.0 / x.v, x.c)


def joint_trig(q):
    n = len(q)
    sq, cq, Sa, Ca = [None] * n, [None] * n, [None] * n, [None] * n
    for i in range(n):
        sq[i], cq[i] = sincos(q[i])
        if i == 0:
            Sa[0], Ca[0] = sq[0], cq[0]
        else:
            Sa[i] = fma(Sa[i - 1], cq[i], Ca[i - 1] * sq[i])
            Ca[i] = fma(Ca[i - 1], cq[i], (-Sa[i - 1]) * sq[i])
    return sq, cq, Sa, Ca


def chain_step(q, v, m, l, b, il, mg, dt):
    """One semi-implicit Euler step of the rank-1 link-frame recursion; returns (q', v')."""
    n = len(q)
    c = q[0].c
    zero = S(0.0, c, True)
    sq, cq, Sa, Ca = joint_trig(q)
    o2, w, tau = [None] * n, [None] * n, [None] * n
    om = zero
    for i in range(n):
        om = om + v[i]
        o2[i] = om * om
        w[i] = o2[i] * l[i]
        tau[i] = (-b[i]) * v[i]
    f, x = [None] * n, [None] * n
    Bce, Bcp, kc = zero, zero, zero
    for i in range(n - 1, -1, -1):
        dtau = fma(-b[i], v[i], -tau[i + 1]) if i + 1 < n else tau[i]
        Be, Bp, h, y, z = zero, zero, m[i], zero, m[i]
        if i + 1 < n:
            s1, c1 = sq[i + 1], cq[i + 1]
            Be = fma(Bce, c1, (-Bcp) * s1)
            Bp = fma(Bce, s1, Bcp * c1)
            ks = kc * s1
            h = fma(ks, s1, m[i])
            y = ks * c1
            z = fma(kc * c1, c1, m[i])
        ih = rcp(h)
        be = fma(-mg[i], Ca[i], fma(-w[i], z, Be))
        bp = fma(mg[i], Sa[i], fma(-w[i], y, Bp))
        ft = fma(dtau, il[i], -bp) * ih
        f[i] = ft
        x[i] = y * ih
        Bce = fma(ft, y, be)
        Bcp = dtau * il[i]
        kc = (m[i] * (m[i] + kc)) * ih
    q2, v2 = list(q), list(v)
    Ae, Ap, alp = zero, zero, zero
    for i in range(n):
        ae, ap = zero, zero
        if i > 0:
            ae = fma(cq[i], Ae, sq[i] * Ap)
            ap = fma(cq[i], Ap, (-sq[i]) * Ae)
        An = fma(-x[i], ae, f[i])
        d = An - ap
        al = d * il[i]
        Ae = fma(-o2[i], l[i], ae)
        Ap = An
        qdd = fma(d, il[i], -alp) if i > 0 else al
        alp = al
        v2[i] = fma(qdd, dt, v2[i])
        q2[i] = fma(v2[i], dt, q2[i])
    return q2, v2


def obs_residual(obs, q, v):
    """sum of r^2 over every state component (the observation term of a step)."""
    c = q[0].c
    acc = S(0.0, c, True)
    state = list(q) + list(v)
    for o, s in zip(obs, state):
        r = o - s
        acc = fma(r, r, acc)
    return acc


def obs_seed(obs, q, v, qb, vb, iso2):
    n = len(q)
    qb, vb = list(qb), list(vb)
    for j in range(n):
        qb[j] = fma(obs[j] - q[j], iso2, qb[j])
        vb[j] = fma(obs[n + j] - v[j], iso2, vb[j])
    return qb, vb


def chain_step_vjp(q, v, v2, m, l, b, il, g, dt, idt, qb, vb, mb, lb, bb, lengths=True):
    """Reverse of one step: (qb, vb) the adjoint of the output state in, that
    of the input state out; mb, lb, bb accumulate the parameter adjoints.
    lengths=False: no link length is a parameter, and the length adjoint
    (p_j.F_j and lb) is not computed; lb comes back unchanged."""
    n = len(q)
    c = q[0].c
    zero = S(0.0, c, True)
    qb, vb, mb, lb, bb = list(qb), list(vb), list(mb), list(lb), list(bb)
    for i in range(n):
        vb[i] = fma(qb[i], dt, vb[i])
    sq, cq, Sa, Ca = joint_trig(q)
    f, x = [None] * n, [None] * n
    Bce, Bcp, kc = zero, zero, zero
    for i in range(n - 1, -1, -1):
        dtau = (vb[i] - vb[i + 1] if i + 1 < n else vb[i]) * dt
        Be, Bp, h, y = zero, zero, m[i], zero
        if i + 1 < n:
            s1, c1 = sq[i + 1], cq[i + 1]
            Be = fma(Bce, c1, (-Bcp) * s1)
            Bp = fma(Bce, s1, Bcp * c1)
            ks = kc * s1
            h = fma(ks, s1, m[i])
            y = ks * c1
        ih = rcp(h)
        ft = fma(dtau, il[i], -Bp) * ih
        f[i] = ft
        x[i] = y * ih
        Bce = fma(ft, y, Be)
        Bcp = dtau * il[i]
        kc = (m[i] * (m[i] + kc)) * ih
    Lam, mu, om, al = [None] * n, [None] * n, [None] * n, [None] * n
    Gx, Gy, dx, dy = [None] * n, [None] * n, [None] * n, [None] * n
    Ae, Ap, o, a, Ax, Ay, ddx, ddy = (zero,) * 8
    for i in range(n):
        ae, ap = zero, zero
        if i > 0:
            ae = fma(cq[i], Ae, sq[i] * Ap)
            ap = fma(cq[i], Ap, (-sq[i]) * Ae)
        An = fma(-x[i], ae, f[i])
        d = An - ap
        Lam[i] = d * il[i]
        mu[i] = fma(d, il[i], -Lam[i - 1]) if i > 0 else Lam[0]
        Ae, Ap = ae, An
        o = o + v[i]
        a = fma(v2[i] - v[i], idt, a)
        om[i], al[i] = o, a
        o2 = o * o
        ux = fma(a, Ca[i], (-o2) * Sa[i])
        uy = fma(a, Sa[i], o2 * Ca[i])
        Ax = fma(l[i], ux, Ax)
        Ay = fma(l[i], uy, Ay)
        ll = l[i] * Lam[i]
        ddx = fma(ll, Ca[i], ddx)
        ddy = fma(ll, Sa[i], ddy)
        Gx[i], Gy[i], dx[i], dy[i] = Ax, Ay + g, ddx, ddy
    m2 = S(-2.0, c)
    Fx, Fy, Dx, Dy, sphi, som = (zero,) * 6
    for i in range(n - 1, -1, -1):
        mi = m[i]
        Fx = fma(mi, Gx[i], Fx)
        Fy = fma(mi, Gy[i], Fy)
        Dx = fma(mi, dx[i], Dx)
        Dy = fma(mi, dy[i], Dy)
        eD = fma(Sa[i], Dx, (-Ca[i]) * Dy)
        pD = fma(Ca[i], Dx, Sa[i] * Dy)
        eF = fma(Sa[i], Fx, (-Ca[i]) * Fy)
        o2 = om[i] * om[i]
        mb[i] = mb[i] - fma(Gx[i], dx[i], Gy[i] * dy[i])
        if lengths:
            pF = fma(Ca[i], Fx, Sa[i] * Fy)
            lb[i] = lb[i] - fma(al[i], pD, fma(-o2, eD, Lam[i] * pF))
        bb[i] = fma(-mu[i], v[i], bb[i])
        som = fma((m2 * om[i]) * l[i], eD, som)
        sphi = fma(l[i], fma(-al[i], eD, fma(-o2, pD, (-Lam[i]) * eF)), sphi)
        qb[i] = qb[i] - sphi
        vb[i] = vb[i] - fma(mu[i], b[i], som)
    return qb, vb, mb, lb, bb
