"""ctypes binding of the FP64 CPU oracle (``oracle/oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this module; the product library never does.

The oracle restates, in double precision and plain loops, what the hot path
computes: planar articulated-body dynamics with semi-implicit Euler
(Appendix B-A, Eq. dynamics), the multiple-shooting likelihood (Sec. IV-C,
Eqs. 2, 4, 5) with the limit prior (Sec. IV-D), its gradient by forward-mode
dual numbers, and the SVGD update (Sec. IV-A, Eq. 1) driven by Adam
(Algorithm 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (g++, -O2, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("g", ctypes.c_double),
        ("mass", _dp),
        ("length", _dp),
        ("damping", _dp),
        ("M", ctypes.c_int),
        ("theta_kind", _ip),
        ("theta_link", _ip),
        ("dt", ctypes.c_double),
        ("T", ctypes.c_int),
        ("W", ctypes.c_int),
        ("D", ctypes.c_int),
        ("obs_index", _ip),
        ("obs", _dp),
        ("sigma_obs", ctypes.c_double),
        ("sigma_def", ctypes.c_double),
        ("s0", _dp),
        ("lo", _dp),
        ("hi", _dp),
        ("c_lim", ctypes.c_double),
        ("R", ctypes.c_int),
        ("combine", ctypes.c_int),
    ]


class _ArmBox(ctypes.Structure):
    _fields_ = [
        ("n_arm", ctypes.c_int),
        ("arm_len", _dp),
        ("amp", _dp),
        ("freq", _dp),
        ("phase", _dp),
        ("box_mass", ctypes.c_double),
        ("box_side", ctypes.c_double),
        ("box_com_depth", ctypes.c_double),
        ("weight_mass0", ctypes.c_double),
        ("weight_mass1", ctypes.c_double),
        ("weight_depth", ctypes.c_double),
        ("g", ctypes.c_double),
        ("damping", ctypes.c_double),
    ]


class _ArmBoxProblem(ctypes.Structure):
    _fields_ = [
        ("ab", _ArmBox),
        ("dt", ctypes.c_double),
        ("T", ctypes.c_int),
        ("W", ctypes.c_int),
        ("D", ctypes.c_int),
        ("obs_index", _ip),
        ("obs", _dp),
        ("sigma_obs", ctypes.c_double),
        ("sigma_def", ctypes.c_double),
        ("s0", _dp),
        ("lo", _dp),
        ("hi", _dp),
        ("c_lim", ctypes.c_double),
    ]


class _Rigid2(ctypes.Structure):
    _fields_ = [("p", ctypes.c_double * 11), ("g", ctypes.c_double)]


class _Rigid2Problem(ctypes.Structure):
    _fields_ = [
        ("sys", _Rigid2),
        ("M", ctypes.c_int),
        ("theta_param", _ip),
        ("dt", ctypes.c_double),
        ("T", ctypes.c_int),
        ("W", ctypes.c_int),
        ("D", ctypes.c_int),
        ("obs_index", _ip),
        ("obs", _dp),
        ("sigma_obs", ctypes.c_double),
        ("sigma_def", ctypes.c_double),
        ("s0", _dp),
        ("lo", _dp),
        ("hi", _dp),
        ("c_lim", ctypes.c_double),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.orc_aba.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_crba.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_fd_crba.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_energy.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp]
            L.orc_energy.restype = ctypes.c_double
            L.orc_simulate.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, ctypes.c_double,
                                       ctypes.c_int, _dp, _dp]
            L.orc_step.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, ctypes.c_double, _dp, _dp]
            L.orc_loglik_grad.argtypes = [ctypes.POINTER(_Problem), _dp, ctypes.c_int, _dp, _dp, ctypes.c_int]
            L.orc_max_threads.restype = ctypes.c_int
            L.orc_median_sqdist.argtypes = [ctypes.c_int, ctypes.c_int, _dp]
            L.orc_median_sqdist.restype = ctypes.c_double
            L.orc_bandwidth.argtypes = [ctypes.c_int, ctypes.c_double]
            L.orc_bandwidth.restype = ctypes.c_double
            L.orc_svgd_phi.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp]
            L.orc_svgd_step.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp,
                                        ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp]
            L.orc_svgd_update.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp,
                                          ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_int]
            L.orc_csvgd_loglik_grad.argtypes = [ctypes.POINTER(_Problem), ctypes.c_double, _dp, ctypes.c_int, _dp,
                                                _dp, ctypes.c_int]
            L.orc_csvgd_step.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp,
                                         _dp, _dp, ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, _dp, _dp]
            L.orc_langevin_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.orc_langevin_normal.restype = ctypes.c_double
            L.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.orc_splitmix64.restype = ctypes.c_uint64
            L.orc_sgld_step.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp,
                                        ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_uint64, ctypes.c_int]
            L.orc_armbox_pivot.argtypes = [ctypes.POINTER(_ArmBox), ctypes.c_double, _dp, _dp]
            L.orc_armbox_qdd.argtypes = [ctypes.POINTER(_ArmBox), _dp, ctypes.c_double, _dp, _dp]
            L.orc_armbox_inertia.argtypes = [ctypes.POINTER(_ArmBox), _dp, _dp]
            L.orc_armbox_simulate.argtypes = [ctypes.POINTER(_ArmBox), _dp, ctypes.c_double, ctypes.c_int, _dp, _dp]
            L.orc_svgd_phi_rows.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double, _ip, ctypes.c_int,
                                            _dp]
            L.orc_rigid2_qdd_full.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp]
            L.orc_rigid2_qdd.argtypes = [_dp, ctypes.c_double, _dp, _dp]
            L.orc_rigid2_simulate.argtypes = [_dp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _dp, _dp]
            L.orc_rigid2_loglik_grad.argtypes = [ctypes.POINTER(_Rigid2Problem), _dp, ctypes.c_int, _dp, _dp,
                                                 ctypes.c_int]
            L.orc_armbox_loglik_grad.argtypes = [ctypes.POINTER(_ArmBoxProblem), _dp, ctypes.c_int, _dp, _dp,
                                                 ctypes.c_int]
            _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


# --------------------------------------------------------------------------
# dynamics
# --------------------------------------------------------------------------
def aba(m, l, b, q, qd, tau, g=9.81):
    """Forward dynamics qdd of the planar point-mass chain by the ABA."""
    n = len(m)
    bufs = [_d(x) for x in (m, l, b, q, qd, tau)]
    out = np.zeros(n)
    lib().orc_aba(n, g, *[p for _, p in bufs], out.ctypes.data_as(_dp))
    return out


def fd_crba(m, l, b, q, qd, tau, g=9.81):
    """Forward dynamics by CRBA + Cholesky (independent of the ABA)."""
    n = len(m)
    bufs = [_d(x) for x in (m, l, b, q, qd, tau)]
    out = np.zeros(n)
    rc = lib().orc_fd_crba(n, g, *[p for _, p in bufs], out.ctypes.data_as(_dp))
    if rc != 0:
        raise RuntimeError("mass matrix not positive definite")
    return out


def crba(m, l, b, q, qd, g=9.81):
    n = len(m)
    bufs = [_d(x) for x in (m, l, b, q, qd)]
    H = np.zeros((n, n))
    C = np.zeros(n)
    lib().orc_crba(n, g, *[p for _, p in bufs], H.ctypes.data_as(_dp), C.ctypes.data_as(_dp))
    return H, C


def energy(m, l, q, qd, g=9.81):
    bufs = [_d(x) for x in (m, l, q, qd)]
    return lib().orc_energy(len(m), g, *[p for _, p in bufs])


def simulate(m, l, b, s0, dt, T, g=9.81):
    """f_sim: states [T+1][2n] from s0 by T semi-implicit Euler steps."""
    n = len(m)
    bufs = [_d(x) for x in (m, l, b, s0)]
    out = np.zeros((T + 1, 2 * n))
    p = [p for _, p in bufs]
    lib().orc_simulate(n, g, p[0], p[1], p[2], dt, T, p[3], out.ctypes.data_as(_dp))
    return out


def step(m, l, b, s, dt, g=9.81):
    n = len(m)
    bufs = [_d(x) for x in (m, l, b, s)]
    out = np.zeros(2 * n)
    p = [p for _, p in bufs]
    lib().orc_step(n, g, p[0], p[1], p[2], dt, p[3], out.ctypes.data_as(_dp))
    return out


# --------------------------------------------------------------------------
# likelihood
# --------------------------------------------------------------------------
class Problem:
    """Multiple-shooting problem for the oracle (all arrays float64/int32).

    ``obs`` is [T][D]: row t-1 holds observation x_t.  Particles are
    [N][P] with P = M + (W-1)*2n: theta first, then s^s_1 .. s^s_{W-1}.
    A set of R trajectories: ``obs`` [R][T][D], ``s0`` [R][2n] and
    ``combine`` "sum" (equally weighted mixture) or "product"; particles then
    carry each trajectory's shooting states in turn, P = M + R (W-1) 2n.
    """

    def __init__(self, *, mass, length, damping, theta_kind, theta_link, dt, T, W, obs, obs_index,
                 sigma_obs, sigma_def, s0, lo, hi, g=9.81, c_lim=1e4, combine="sum"):
        self._keep = []

        def d(x):
            a, p = _d(x)
            self._keep.append(a)
            return p

        def i(x):
            a, p = _i(x)
            self._keep.append(a)
            return p

        self.n = len(mass)
        self.M = len(theta_kind)
        self.W = int(W)
        self.T = int(T)
        self.S = 2 * self.n
        obs = np.asarray(obs, dtype=np.float64)
        s0 = np.asarray(s0, dtype=np.float64)
        if obs.ndim == 2:
            obs, s0 = obs[None], s0.reshape(1, -1)
        self.R = obs.shape[0]
        assert s0.shape == (self.R, self.S) and combine in ("sum", "product")
        self.P = self.M + self.R * (self.W - 1) * self.S
        self.D = obs.shape[2]
        self.c = _Problem(
            n=self.n, g=float(g), mass=d(mass), length=d(length), damping=d(damping), M=self.M,
            theta_kind=i(theta_kind), theta_link=i(theta_link), dt=float(dt), T=self.T, W=self.W, D=self.D,
            obs_index=i(obs_index), obs=d(obs), sigma_obs=float(sigma_obs), sigma_def=float(sigma_def),
            s0=d(s0), lo=d(lo), hi=d(hi), c_lim=float(c_lim), R=self.R, combine=0 if combine == "sum" else 1)

    @property
    def Pc(self):
        """Particle length of the constrained method: theta, shooting states,
        the W-1 defect multipliers and the M limit multipliers."""
        return self.P + (self.W - 1) + self.M

    def csvgd_loglik_grad(self, particles, c=1.0, threads=1):
        """Constrained SVGD (Sec. IV-E): returns (log p_obs [N], out [N][Pc+M])
        with out's rows as orc_csvgd_loglik_grad documents: d log p_obs/d theta,
        d(log p_obs - Psi)/d s^s, g_def, g_lim, -dPsi/d theta."""
        assert self.R == 1, "constrained SVGD is built for one trajectory"
        x, xp = _d(np.atleast_2d(particles))
        N = x.shape[0]
        assert x.shape[1] == self.Pc, (x.shape, self.Pc)
        logp = np.zeros(N)
        out = np.zeros((N, self.Pc + self.M))
        rc = lib().orc_csvgd_loglik_grad(ctypes.byref(self.c), float(c), xp, N, logp.ctypes.data_as(_dp),
                                         out.ctypes.data_as(_dp), int(threads))
        if rc != 0:
            raise RuntimeError(f"orc_csvgd_loglik_grad failed ({rc})")
        return logp, out

    def loglik_grad(self, particles, grad=True, threads=1):
        x, xp = _d(np.atleast_2d(particles))
        N = x.shape[0]
        assert x.shape[1] == self.P, (x.shape, self.P)
        logp = np.zeros(N)
        g = np.zeros((N, self.P)) if grad else None
        rc = lib().orc_loglik_grad(ctypes.byref(self.c), xp, N, logp.ctypes.data_as(_dp),
                                   g.ctypes.data_as(_dp) if grad else None, int(threads))
        if rc != 0:
            raise RuntimeError(f"orc_loglik_grad failed ({rc})")
        return (logp, g) if grad else logp


def max_threads() -> int:
    return int(lib().orc_max_threads())


# --------------------------------------------------------------------------
# SVGD
# --------------------------------------------------------------------------
def splitmix64(seed: int, index: int) -> int:
    """Output `index` (1-based) of the SplitMix64 sequence from `seed`."""
    return lib().orc_splitmix64(int(seed), int(index))


def langevin_normal(seed: int, k: int) -> float:
    """The SGLD noise generator's standard normal number k for `seed`."""
    return lib().orc_langevin_normal(int(seed), int(k))


class SgldState:
    """Step count of the oracle's SGLD chains (one chain per particle)."""

    def __init__(self, N, P, lo, hi, a=1e-4, b=1.0, gamma=0.55, seed=0, clamp=True):
        self.N, self.P = N, P
        self.M = len(lo)
        self.lo = np.ascontiguousarray(lo, dtype=np.float64)
        self.hi = np.ascontiguousarray(hi, dtype=np.float64)
        self.t = ctypes.c_int(0)
        self.a, self.b, self.gamma, self.seed, self.clamp = a, b, gamma, seed, clamp

    def step(self, particles, grad):
        """In-place SGLD update of particles [N][P] with gradient [N][P]."""
        assert particles.dtype == np.float64 and particles.flags.c_contiguous
        g, gp = _d(grad)
        lib().orc_sgld_step(self.N, self.M, self.P, self.lo.ctypes.data_as(_dp), self.hi.ctypes.data_as(_dp),
                            particles.ctypes.data_as(_dp), gp, ctypes.byref(self.t), float(self.a), float(self.b),
                            float(self.gamma), int(self.seed), int(self.clamp))


class CsvgdState:
    """Adam moments and step count of the oracle's constrained SVGD update
    (Algorithm 1): particles [N][Pc] with Pc = M + n_shoot + n_def + M."""

    def __init__(self, N, Pc, n_def, lo, hi, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
        self.N, self.Pc, self.n_def = N, Pc, n_def
        self.M = len(lo)
        self.lo = np.ascontiguousarray(lo, dtype=np.float64)
        self.hi = np.ascontiguousarray(hi, dtype=np.float64)
        self.m = np.zeros((N, Pc))
        self.v = np.zeros((N, Pc))
        self.t = ctypes.c_int(0)
        self.lr, self.beta1, self.beta2, self.eps = lr, beta1, beta2, eps

    def step(self, particles, out):
        """In-place update of particles [N][Pc] from out [N][Pc+M]; returns (phi, bw)."""
        assert particles.dtype == np.float64 and particles.flags.c_contiguous
        o, op = _d(out)
        assert o.shape == (self.N, self.Pc + self.M)
        phi = np.zeros((self.N, self.M))
        bw = ctypes.c_double(0.0)
        rc = lib().orc_csvgd_step(self.N, self.M, self.Pc, self.n_def, self.lo.ctypes.data_as(_dp),
                                  self.hi.ctypes.data_as(_dp), particles.ctypes.data_as(_dp), op,
                                  self.m.ctypes.data_as(_dp), self.v.ctypes.data_as(_dp), ctypes.byref(self.t),
                                  self.lr, self.beta1, self.beta2, self.eps, phi.ctypes.data_as(_dp),
                                  ctypes.byref(bw))
        if rc != 0:
            raise RuntimeError("orc_csvgd_step failed")
        return phi, bw.value

def median_sqdist(u):
    u, up = _d(np.atleast_2d(u))
    return lib().orc_median_sqdist(u.shape[0], u.shape[1], up)


def bandwidth(N, med):
    return lib().orc_bandwidth(int(N), float(med))


def svgd_phi(u, g, bw):
    u, up = _d(u)
    g, gp = _d(g)
    out = np.zeros_like(u)
    lib().orc_svgd_phi(u.shape[0], u.shape[1], up, gp, float(bw), out.ctypes.data_as(_dp))
    return out


def svgd_phi_rows(u, g, bw, rows):
    """phi (Eq. 1) of the particles `rows` only, [len(rows)][M]."""
    u, up = _d(u)
    g, gp = _d(g)
    r, rp = _i(rows)
    out = np.zeros((len(r), u.shape[1]))
    rc = lib().orc_svgd_phi_rows(u.shape[0], u.shape[1], up, gp, float(bw), rp, len(r), out.ctypes.data_as(_dp))
    if rc != 0:
        raise ValueError("row index out of range")
    return out


class SvgdState:
    """Adam moments and step count of the oracle's SVGD iteration."""

    def __init__(self, N, P, lo, hi, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, clamp=True):
        self.N, self.P = N, P
        self.M = len(lo)
        self.lo = np.ascontiguousarray(lo, dtype=np.float64)
        self.hi = np.ascontiguousarray(hi, dtype=np.float64)
        self.m = np.zeros((N, P))
        self.v = np.zeros((N, P))
        self.t = ctypes.c_int(0)
        self.lr, self.beta1, self.beta2, self.eps, self.clamp = lr, beta1, beta2, eps, clamp

    def step(self, particles, grad):
        """In-place SVGD+Adam update of particles [N][P]; returns (phi, bw)."""
        assert particles.dtype == np.float64 and particles.flags.c_contiguous
        g, gp = _d(grad)
        phi = np.zeros((self.N, self.M))
        bw = ctypes.c_double(0.0)
        lib().orc_svgd_step(self.N, self.M, self.P, self.lo.ctypes.data_as(_dp), self.hi.ctypes.data_as(_dp),
                            particles.ctypes.data_as(_dp), gp, self.m.ctypes.data_as(_dp),
                            self.v.ctypes.data_as(_dp), ctypes.byref(self.t), self.lr, self.beta1, self.beta2,
                            self.eps, int(self.clamp), phi.ctypes.data_as(_dp), ctypes.byref(bw))
        return phi, bw.value

    def update(self, particles, phi, grad):
        """The update half of ``step`` with given directions: Adam ascent of
        the theta rows on phi [N][M] (unit-box coordinates) and of the
        shooting-state rows on grad [N][P] (Algorithm 1)."""
        assert particles.dtype == np.float64 and particles.flags.c_contiguous
        ph, pp = _d(phi)
        g, gp = _d(grad)
        lib().orc_svgd_update(self.N, self.M, self.P, self.lo.ctypes.data_as(_dp), self.hi.ctypes.data_as(_dp),
                              particles.ctypes.data_as(_dp), pp, gp, self.m.ctypes.data_as(_dp),
                              self.v.ctypes.data_as(_dp), ctypes.byref(self.t), self.lr, self.beta1, self.beta2,
                              self.eps, int(self.clamp))


# --------------------------------------------------------------------------
# arm shaking a box
# --------------------------------------------------------------------------
class ArmBox:
    """Prescribed arm + U-joint box description (see oracle.cpp)."""

    def __init__(self, *, arm_len, amp, freq, phase, box_mass=1.0, box_side=0.3, box_com_depth=0.15,
                 weight_mass=(0.5, 0.5), weight_depth=0.3, g=9.81, damping=0.0):
        self._keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (arm_len, amp, freq, phase)]
        a, b, c, d = self._keep
        self.c = _ArmBox(n_arm=len(a), arm_len=a.ctypes.data_as(_dp), amp=b.ctypes.data_as(_dp),
                         freq=c.ctypes.data_as(_dp), phase=d.ctypes.data_as(_dp), box_mass=box_mass,
                         box_side=box_side, box_com_depth=box_com_depth, weight_mass0=weight_mass[0],
                         weight_mass1=weight_mass[1], weight_depth=weight_depth, g=g, damping=damping)

    @classmethod
    def from_workload(cls, wl):
        return cls(arm_len=wl.arm_len, amp=wl.amp, freq=wl.freq, phase=wl.phase, box_mass=wl.box_mass,
                   box_side=wl.box_side, box_com_depth=wl.box_com_depth, weight_mass=wl.weight_mass,
                   weight_depth=wl.weight_depth, g=wl.g, damping=wl.box_damping)

    def pivot(self, t):
        v, a = np.zeros(6), np.zeros(6)
        lib().orc_armbox_pivot(ctypes.byref(self.c), float(t), v.ctypes.data_as(_dp), a.ctypes.data_as(_dp))
        return v, a

    def qdd(self, theta, t, s):
        th, tp = _d(theta)
        st, sp = _d(s)
        out = np.zeros(2)
        lib().orc_armbox_qdd(ctypes.byref(self.c), tp, float(t), sp, out.ctypes.data_as(_dp))
        return out

    def inertia(self, theta):
        th, tp = _d(theta)
        out = np.zeros((6, 6))
        lib().orc_armbox_inertia(ctypes.byref(self.c), tp, out.ctypes.data_as(_dp))
        return out

    def simulate(self, theta, dt, T, s0):
        th, tp = _d(theta)
        s, sp = _d(s0)
        out = np.zeros((T + 1, 4))
        lib().orc_armbox_simulate(ctypes.byref(self.c), tp, float(dt), int(T), sp, out.ctypes.data_as(_dp))
        return out


class ArmBoxProblem:
    """Multiple-shooting problem of the box (theta = (x1, y1, x2, y2))."""

    def __init__(self, armbox: ArmBox, *, dt, T, W, obs, obs_index, sigma_obs, sigma_def, s0, lo, hi, c_lim=1e4):
        self.armbox = armbox
        self._keep = []

        def d(x):
            a, p = _d(x)
            self._keep.append(a)
            return p

        def i(x):
            a, p = _i(x)
            self._keep.append(a)
            return p

        obs = np.asarray(obs, dtype=np.float64)
        self.T, self.W, self.M, self.S = int(T), int(W), 4, 4
        self.P = 4 + (self.W - 1) * 4
        self.c = _ArmBoxProblem(ab=armbox.c, dt=float(dt), T=self.T, W=self.W, D=obs.shape[1], obs_index=i(obs_index),
                                obs=d(obs), sigma_obs=float(sigma_obs), sigma_def=float(sigma_def), s0=d(s0),
                                lo=d(lo), hi=d(hi), c_lim=float(c_lim))

    def loglik_grad(self, particles, grad=True, threads=1):
        x, xp = _d(np.atleast_2d(particles))
        N = x.shape[0]
        assert x.shape[1] == self.P
        logp = np.zeros(N)
        g = np.zeros((N, self.P)) if grad else None
        rc = lib().orc_armbox_loglik_grad(ctypes.byref(self.c), xp, N, logp.ctypes.data_as(_dp),
                                          g.ctypes.data_as(_dp) if grad else None, int(threads))
        if rc != 0:
            raise RuntimeError("orc_armbox_loglik_grad failed")
        return (logp, g) if grad else logp


# --------------------------------------------------------------------------
# Rigid double pendulum (11 parameters: [m1, I1, c1x, c1y, b1, l, m2, I2,
# c2x, c2y, b2]; joints about z, joint 2 at (0, -l, 0) in link 1's frame,
# gravity along -y; state [q1, q2, qd1, qd2])
# --------------------------------------------------------------------------
RIGID2_PARAMS = ("m1", "I1", "c1x", "c1y", "b1", "l", "m2", "I2", "c2x", "c2y", "b2")


def rigid2_qdd_full(m, c, Ic, b, l, g, s):
    """Joint accelerations for general COMs c [2][3] and inertias Ic [2][3][3]."""
    ma, mp = _d(m)
    ca, cp = _d(np.asarray(c, dtype=np.float64).reshape(-1))
    ia, ip = _d(np.asarray(Ic, dtype=np.float64).reshape(-1))
    ba, bp = _d(b)
    sa, sp = _d(s)
    out = np.zeros(2)
    lib().orc_rigid2_qdd_full(mp, cp, ip, bp, float(l), float(g), sp, out.ctypes.data_as(_dp))
    return out


def rigid2_qdd(p11, g, s):
    pa, pp = _d(p11)
    sa, sp = _d(s)
    out = np.zeros(2)
    lib().orc_rigid2_qdd(pp, float(g), sp, out.ctypes.data_as(_dp))
    return out


def rigid2_simulate(p11, g, dt, T, s0):
    pa, pp = _d(p11)
    sa, sp = _d(s0)
    out = np.zeros((T + 1, 4))
    lib().orc_rigid2_simulate(pp, float(g), float(dt), int(T), sp, out.ctypes.data_as(_dp))
    return out


class Rigid2Problem:
    """Multiple-shooting problem of the rigid double pendulum: theta are the
    parameters theta_param (indices into the 11), the others fixed at p11."""

    def __init__(self, *, p11, g, theta_param, dt, T, W, obs, obs_index, sigma_obs, sigma_def, s0, lo, hi,
                 c_lim=1e4):
        self._keep = []

        def d(x):
            a, p = _d(x)
            self._keep.append(a)
            return p

        def i(x):
            a, p = _i(x)
            self._keep.append(a)
            return p

        obs = np.asarray(obs, dtype=np.float64)
        self.T, self.W, self.M, self.S = int(T), int(W), len(theta_param), 4
        self.P = self.M + (self.W - 1) * 4
        sysc = _Rigid2(g=float(g))
        for k in range(11):
            sysc.p[k] = float(p11[k])
        self.c = _Rigid2Problem(sys=sysc, M=self.M, theta_param=i(theta_param), dt=float(dt), T=self.T, W=self.W,
                                D=obs.shape[1], obs_index=i(obs_index), obs=d(obs), sigma_obs=float(sigma_obs),
                                sigma_def=float(sigma_def), s0=d(s0), lo=d(lo), hi=d(hi), c_lim=float(c_lim))

    def loglik_grad(self, particles, grad=True, threads=1):
        x, xp = _d(np.atleast_2d(particles))
        N = x.shape[0]
        assert x.shape[1] == self.P
        logp = np.zeros(N)
        g = np.zeros((N, self.P)) if grad else None
        rc = lib().orc_rigid2_loglik_grad(ctypes.byref(self.c), xp, N, logp.ctypes.data_as(_dp),
                                          g.ctypes.data_as(_dp) if grad else None, int(threads))
        if rc != 0:
            raise RuntimeError("orc_rigid2_loglik_grad failed")
        return (logp, g) if grad else logp
