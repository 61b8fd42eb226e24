"""Seeded synthetic workloads shaped like the paper's experiments.

This module holds random draws and configuration constants only: no dynamics,
no likelihood, no SVGD arithmetic.  It is the one module that both the CUDA
path (through the Python binding) and the FP64 oracle (in the tests) take
their inputs from, so that the two sides see identical arrays.

Observations are produced by whoever rolls out the true parameters (the
oracle in tests, the library's own ``simulate`` in the benchmark); this module
only supplies the true parameters, the initial state and the standard-normal
noise draws that are scaled by sigma_obs.

Workloads (synthetic stand-ins; the paper's real datasets are not available):

* ``double_pendulum`` -- the paper's double-pendulum setting (Sec. V-A, V-B):
  2 revolute links, theta = (m1, m2, l1, l2), 200 steps at dt = 0.01,
  angles observed with sigma 0.01, 10 shooting windows, 100 particles.
* ``chain5`` -- a 5-link planar chain with point masses at the link tips and
  viscous joint damping, theta = 5 masses + 5 damping coefficients, 1000 steps
  at dt = 0.005, angles and velocities observed with sigma 0.02, 20 windows.
* ``rigid_double_pendulum`` -- the physical double pendulum's 11-parameter
  rigid-body model (masses, inertias, centres of mass, joint frictions, the
  second joint's offset) at 400 Hz, 1000 steps, 10 windows.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

PARAM_MASS = 0
PARAM_LENGTH = 1
PARAM_DAMPING = 2

GRAVITY = 9.81
SIGMA_DEF = 0.1          # sigma_def^2 = 1e-2, the "small variance" of Eq. 4
C_LIM = 1.0e4            # stiffness of the smooth parameter-limit penalty


@dataclasses.dataclass
class PlanarWorkload:
    name: str
    n: int
    mass: np.ndarray            # [n] true masses (theta entries override)
    length: np.ndarray          # [n]
    damping: np.ndarray         # [n]
    theta_kind: np.ndarray      # [M] int32, PARAM_*
    theta_link: np.ndarray      # [M] int32
    theta_true: np.ndarray      # [M]
    lo: np.ndarray              # [M] prior box
    hi: np.ndarray              # [M]
    dt: float
    T: int
    W: int
    obs_index: np.ndarray       # [D] int32 indices into s = [q, qd]
    sigma_obs: float
    sigma_def: float
    s0: np.ndarray              # [2n]
    noise: np.ndarray           # [T][D] standard normal draws
    theta_init: np.ndarray      # [N][M] initial particles, uniform in the box
    lr: float = 1e-2
    iterations: int = 100
    g: float = GRAVITY
    c_lim: float = C_LIM
    seed: int = 0

    @property
    def M(self) -> int:
        return len(self.theta_kind)

    @property
    def S(self) -> int:
        return 2 * self.n

    @property
    def D(self) -> int:
        return len(self.obs_index)

    @property
    def N(self) -> int:
        return self.theta_init.shape[0]

    @property
    def P(self) -> int:
        return self.M + (self.W - 1) * self.S

    def window_start(self, w: int) -> int:
        return (w * self.T) // self.W


def double_pendulum(N: int = 100, seed: int = 1000) -> PlanarWorkload:
    """Double pendulum, theta = (m1, m2, l1, l2).

    True masses ~ U[0.5, 2], lengths ~ U[0.5, 1.5]; q0 ~ U(-pi/2, pi/2),
    zero velocity; no damping.  The prior box is the sampling box.
    """
    rng = np.random.default_rng(seed)
    lo = np.array([0.5, 0.5, 0.5, 0.5])
    hi = np.array([2.0, 2.0, 1.5, 1.5])
    theta_true = rng.uniform(lo, hi)
    q0 = rng.uniform(-math.pi / 2, math.pi / 2, size=2)
    T, D = 200, 2
    noise = rng.standard_normal((T, D))
    theta_init = rng.uniform(lo, hi, size=(N, 4))
    return PlanarWorkload(
        name="double_pendulum", n=2,
        mass=theta_true[:2].copy(), length=theta_true[2:].copy(), damping=np.zeros(2),
        theta_kind=np.array([PARAM_MASS, PARAM_MASS, PARAM_LENGTH, PARAM_LENGTH], dtype=np.int32),
        theta_link=np.array([0, 1, 0, 1], dtype=np.int32),
        theta_true=theta_true, lo=lo, hi=hi, dt=0.01, T=T, W=10,
        obs_index=np.array([0, 1], dtype=np.int32), sigma_obs=0.01, sigma_def=SIGMA_DEF,
        s0=np.concatenate([q0, np.zeros(2)]), noise=noise, theta_init=theta_init,
        lr=1e-2, iterations=100, seed=seed)


def two_mode_pendulums(N: int = 100, seed: int = 6000):
    """Two double-pendulum trajectories from two different link-length
    settings (the setting of the paper's combination figure): unit masses,
    theta = (l1, l2) in [0.5, 1.5]^2, both started at q0 = (90 deg, 0 deg) at
    rest, 300 steps of 0.01 s, angles observed with sigma 0.01, 10 windows.

    Returns (workload, [theta_a, theta_b], [noise_a, noise_b]): the workload
    carries theta_a as theta_true and noise_a; noise_b is the second
    trajectory's standard-normal observation noise [T][D].
    """
    rng = np.random.default_rng(seed)
    lo = np.array([0.5, 0.5])
    hi = np.array([1.5, 1.5])
    theta_a = np.array([0.7, 1.2])
    theta_b = np.array([1.2, 0.7])
    T, D = 300, 2
    noise = [rng.standard_normal((T, D)) for _ in range(2)]
    theta_init = rng.uniform(lo, hi, size=(N, 2))
    wl = PlanarWorkload(
        name="two_mode_pendulums", n=2, mass=np.ones(2), length=theta_a.copy(), damping=np.zeros(2),
        theta_kind=np.array([PARAM_LENGTH, PARAM_LENGTH], dtype=np.int32),
        theta_link=np.array([0, 1], dtype=np.int32), theta_true=theta_a, lo=lo, hi=hi, dt=0.01, T=T, W=10,
        obs_index=np.array([0, 1], dtype=np.int32), sigma_obs=0.01, sigma_def=SIGMA_DEF,
        s0=np.array([math.pi / 2, 0.0, 0.0, 0.0]), noise=noise[0], theta_init=theta_init,
        lr=1e-2, iterations=300, seed=seed)
    return wl, [theta_a, theta_b], noise


CHAIN5_LENGTH = 0.5      # fixed link length [m]; lengths are not inferred


def chain5(N: int = 1024, seed: int | None = None, T: int = 1000, W: int = 20) -> PlanarWorkload:
    """5-link damped chain, theta = 5 masses + 5 damping coefficients ~ U[0.1, 2].

    Fixed link lengths 0.5 m; q0 ~ U(-pi/2, pi/2) relative angles, zero
    velocity; angles and velocities observed with sigma 0.02.
    """
    if seed is None:
        seed = 2000 + N
    rng = np.random.default_rng(seed)
    n = 5
    lo = np.full(2 * n, 0.1)
    hi = np.full(2 * n, 2.0)
    theta_true = rng.uniform(lo, hi)
    q0 = rng.uniform(-math.pi / 2, math.pi / 2, size=n)
    D = 2 * n
    noise = rng.standard_normal((T, D))
    theta_init = rng.uniform(lo, hi, size=(N, 2 * n))
    kind = np.array([PARAM_MASS] * n + [PARAM_DAMPING] * n, dtype=np.int32)
    link = np.array(list(range(n)) * 2, dtype=np.int32)
    return PlanarWorkload(
        name="chain5", n=n,
        mass=theta_true[:n].copy(), length=np.full(n, CHAIN5_LENGTH), damping=theta_true[n:].copy(),
        theta_kind=kind, theta_link=link, theta_true=theta_true, lo=lo, hi=hi, dt=0.005, T=T, W=W,
        obs_index=np.arange(D, dtype=np.int32), sigma_obs=0.02, sigma_def=SIGMA_DEF,
        s0=np.concatenate([q0, np.zeros(n)]), noise=noise, theta_init=theta_init,
        lr=1e-2, iterations=100, seed=seed)


def random_chain(n: int, N: int, seed: int, T: int = 40, W: int = 4, kinds=(PARAM_MASS, PARAM_LENGTH, PARAM_DAMPING),
                 dt: float = 0.005, observe_velocity: bool = True) -> PlanarWorkload:
    """Small random chain used by parity tests (all three parameter kinds)."""
    rng = np.random.default_rng(seed)
    ranges = {PARAM_MASS: (0.3, 2.0), PARAM_LENGTH: (0.3, 1.2), PARAM_DAMPING: (0.0, 0.8)}
    kind, link, lo, hi = [], [], [], []
    for k in kinds:
        for i in range(n):
            kind.append(k)
            link.append(i)
            lo.append(ranges[k][0])
            hi.append(ranges[k][1])
    lo, hi = np.array(lo), np.array(hi)
    theta_true = rng.uniform(lo, hi)
    mass = rng.uniform(0.3, 2.0, n)
    length = rng.uniform(0.3, 1.2, n)
    damping = rng.uniform(0.0, 0.8, n)
    for j, (k, i) in enumerate(zip(kind, link)):
        {PARAM_MASS: mass, PARAM_LENGTH: length, PARAM_DAMPING: damping}[k][i] = theta_true[j]
    q0 = rng.uniform(-math.pi / 2, math.pi / 2, size=n)
    qd0 = rng.uniform(-1.0, 1.0, size=n)
    obs_index = np.arange(2 * n if observe_velocity else n, dtype=np.int32)
    noise = rng.standard_normal((T, len(obs_index)))
    theta_init = rng.uniform(lo, hi, size=(N, len(kind)))
    return PlanarWorkload(
        name=f"chain{n}", n=n, mass=mass, length=length, damping=damping,
        theta_kind=np.array(kind, dtype=np.int32), theta_link=np.array(link, dtype=np.int32),
        theta_true=theta_true, lo=lo, hi=hi, dt=dt, T=T, W=W, obs_index=obs_index,
        sigma_obs=0.02, sigma_def=SIGMA_DEF, s0=np.concatenate([q0, qd0]), noise=noise,
        theta_init=theta_init, seed=seed)


def observations(wl: PlanarWorkload, states: np.ndarray) -> np.ndarray:
    """x_t = (observed components of s_t) + sigma_obs * noise_t, t = 1..T.

    ``states`` is the true rollout [T+1][2n] (row 0 = s_0).  Returns [T][D].
    """
    return states[1:, wl.obs_index] + wl.sigma_obs * wl.noise


def initial_particles(wl: PlanarWorkload, obs: np.ndarray, N: int | None = None, rng_seed: int | None = None
                      ) -> np.ndarray:
    """Initial augmented particles [N][P] (theta, then s^s_1..s^s_{W-1}).

    theta: the workload's uniform draws in the prior box.  Shooting states:
    the observed components at t_w; unobserved velocities from central
    differences of the observed angles (as for the real pendulum data in
    Appendix B-B).  Identical for all particles.
    """
    theta = wl.theta_init if N is None else wl.theta_init[:N]
    N = theta.shape[0]
    S, n = wl.S, wl.n
    shoot = np.zeros((wl.W - 1, S))
    for w in range(1, wl.W):
        t = wl.window_start(w)
        row = obs[t - 1]
        for d, idx in enumerate(wl.obs_index):
            shoot[w - 1, idx] = row[d]
        for i in range(n):
            if (n + i) not in set(int(x) for x in wl.obs_index):
                d = list(int(x) for x in wl.obs_index).index(i)
                nxt = obs[min(t, wl.T - 1), d]
                prv = obs[max(t - 2, 0), d]
                shoot[w - 1, n + i] = (nxt - prv) / (2.0 * wl.dt)
    x = np.zeros((N, wl.P))
    x[:, :wl.M] = theta
    x[:, wl.M:] = shoot.reshape(-1)[None, :]
    if rng_seed is not None:
        rng = np.random.default_rng(rng_seed)
        x[:, wl.M:] += 0.05 * rng.standard_normal((N, wl.P - wl.M))
    return x


def batched_problems(n_jobs: int = 64, seed: int = 4000, n_range=(2, 8), T_range=(100, 2000), W_range=(5, 50),
                     N_range=(64, 4096)) -> list[PlanarWorkload]:
    """Independent problems of uneven size for batched execution.

    Chain length n ~ U{2..8}; T, W and N log-uniform in their ranges (W at
    most T/2); parameter types of the double pendulum (masses + lengths,
    dt = 0.01, angles observed, sigma 0.01) or of the damped chain (masses +
    damping, dt = 0.005, angles and velocities observed, sigma 0.02), 50/50.
    """
    rng = np.random.default_rng(seed)

    def logu(lo, hi):
        return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))

    out = []
    for j in range(n_jobs):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        T = logu(*T_range)
        W = max(1, min(logu(*W_range), T // 2))
        N = logu(*N_range)
        pend = bool(rng.uniform() < 0.5)
        if pend:
            lo = np.concatenate([np.full(n, 0.5), np.full(n, 0.5)])
            hi = np.concatenate([np.full(n, 2.0), np.full(n, 1.5)])
            kind = [PARAM_MASS] * n + [PARAM_LENGTH] * n
            dt, sig = 0.01, 0.01
            obs_index = np.arange(n, dtype=np.int32)
        else:
            lo = np.full(2 * n, 0.1)
            hi = np.full(2 * n, 2.0)
            kind = [PARAM_MASS] * n + [PARAM_DAMPING] * n
            dt, sig = 0.005, 0.02
            obs_index = np.arange(2 * n, dtype=np.int32)
        theta_true = rng.uniform(lo, hi)
        mass = theta_true[:n].copy()
        length = theta_true[n:].copy() if pend else np.full(n, CHAIN5_LENGTH)
        damping = np.zeros(n) if pend else theta_true[n:].copy()
        q0 = rng.uniform(-math.pi / 2, math.pi / 2, size=n)
        noise = rng.standard_normal((T, len(obs_index)))
        theta_init = rng.uniform(lo, hi, size=(N, 2 * n))
        out.append(PlanarWorkload(
            name=f"batch{j}_{'pend' if pend else 'damped'}{n}", n=n, mass=mass, length=length, damping=damping,
            theta_kind=np.array(kind, dtype=np.int32), theta_link=np.array(list(range(n)) * 2, dtype=np.int32),
            theta_true=theta_true, lo=lo, hi=hi, dt=dt, T=T, W=W, obs_index=obs_index, sigma_obs=sig,
            sigma_def=SIGMA_DEF, s0=np.concatenate([q0, np.zeros(n)]), noise=noise, theta_init=theta_init,
            lr=1e-2, seed=seed + j))
    return out


@dataclasses.dataclass
class ArmBoxWorkload:
    """Arm shaking a box (the paper's Panda-arm experiment, Sec. V-C, synthetic).

    A serial arm of revolute joints (axes alternate z, y, z, ...; link i
    offset l_i along its local z) follows prescribed joint trajectories
    q_j(t) = sum_k amp_jk sin(2 pi f_jk t + phase_jk).  A cube of side 0.3 m
    and mass 1 kg (COM 0.15 m below the joint) hangs from the arm's tip on a
    U-joint (axis x, then y); two 0.5 kg point weights sit on its floor at
    (x_k, y_k, -0.3).  theta = (x1, y1, x2, y2).  The box joint angles are
    observed.
    """
    name: str
    arm_len: np.ndarray        # [n_arm]
    arm_mass: np.ndarray       # [n_arm] (the arm's motion is prescribed; kept for completeness)
    amp: np.ndarray            # [n_arm][3]
    freq: np.ndarray           # [n_arm][3]
    phase: np.ndarray          # [n_arm][3]
    theta_true: np.ndarray     # [4]
    lo: np.ndarray
    hi: np.ndarray
    dt: float
    T: int
    W: int
    obs_index: np.ndarray
    sigma_obs: float
    sigma_def: float
    s0: np.ndarray             # [4]
    noise: np.ndarray          # [T][D]
    theta_init: np.ndarray     # [N][4]
    box_mass: float = 1.0
    box_side: float = 0.3
    box_com_depth: float = 0.15
    weight_mass: tuple = (0.5, 0.5)
    weight_depth: float = 0.3
    box_damping: float = 0.0
    g: float = GRAVITY
    c_lim: float = C_LIM
    lr: float = 1e-2
    iterations: int = 500
    seed: int = 0
    n: int = 2
    M: int = 4
    S: int = 4

    @property
    def D(self) -> int:
        return len(self.obs_index)

    @property
    def N(self) -> int:
        return self.theta_init.shape[0]

    @property
    def P(self) -> int:
        return self.M + (self.W - 1) * self.S

    def window_start(self, w: int) -> int:
        return (w * self.T) // self.W


def arm_box(N: int = 2048, seed: int = 3000, T: int = 2000, W: int = 40, n_arm: int = 7) -> ArmBoxWorkload:
    """7-joint arm (lengths U[0.1, 0.4] m, masses U[1, 4] kg), each joint a sum
    of 3 sinusoids of amplitude 0.3 rad and frequency U[0.2, 1] Hz; weight
    positions ~ U[-0.15, 0.15]; T = 2000 at dt = 0.002, 40 windows, box
    angles observed with sigma 0.01; the box starts at rest in the tip frame."""
    rng = np.random.default_rng(seed)
    arm_len = rng.uniform(0.1, 0.4, n_arm)
    arm_mass = rng.uniform(1.0, 4.0, n_arm)
    amp = np.full((n_arm, 3), 0.3)
    freq = rng.uniform(0.2, 1.0, (n_arm, 3))
    phase = rng.uniform(0.0, 2 * math.pi, (n_arm, 3))
    lo, hi = np.full(4, -0.15), np.full(4, 0.15)
    theta_true = rng.uniform(lo, hi)
    obs_index = np.array([0, 1], dtype=np.int32)
    noise = rng.standard_normal((T, 2))
    theta_init = rng.uniform(lo, hi, size=(N, 4))
    return ArmBoxWorkload(name="arm_box", arm_len=arm_len, arm_mass=arm_mass, amp=amp, freq=freq, phase=phase,
                          theta_true=theta_true, lo=lo, hi=hi, dt=0.002, T=T, W=W, obs_index=obs_index,
                          sigma_obs=0.01, sigma_def=SIGMA_DEF, s0=np.zeros(4), noise=noise, theta_init=theta_init,
                          seed=seed)


RIGID2_PARAMS = ("m1", "I1", "c1x", "c1y", "b1", "l", "m2", "I2", "c2x", "c2y", "b2")
# parameter limits of the physical double pendulum's table (link 1: mass,
# inertia, COM x, COM y, joint friction; link 2: length, mass, inertia, COM x,
# COM y, joint friction)
RIGID2_LO = np.array([0.05, 0.002, -0.2, -0.2, 0.0, 0.08, 0.05, 0.002, -0.2, -0.2, 0.0])
RIGID2_HI = np.array([0.5, 1.0, 0.2, 0.2, 0.5, 0.3, 0.5, 1.0, 0.2, 0.2, 0.5])


@dataclasses.dataclass
class Rigid2Workload:
    """Rigid double pendulum with general inertia and centre of mass (the
    11-parameter physical double pendulum, synthetic): parameters
    [m1, I1, c1x, c1y, b1, l, m2, I2, c2x, c2y, b2]; theta_param selects the
    estimated ones, the others stay at p11."""
    name: str
    p11: np.ndarray            # [11] true values of all parameters
    theta_param: np.ndarray    # [M] int32 indices into p11
    theta_true: np.ndarray     # [M]
    lo: np.ndarray             # [M]
    hi: np.ndarray             # [M]
    dt: float
    T: int
    W: int
    obs_index: np.ndarray      # [D] int32 into s = [q1, q2, qd1, qd2]
    sigma_obs: float
    sigma_def: float
    s0: np.ndarray             # [4]
    noise: np.ndarray          # [T][D]
    theta_init: np.ndarray     # [N][M]
    g: float = GRAVITY
    c_lim: float = C_LIM
    lr: float = 1e-2
    iterations: int = 2000
    seed: int = 0
    n: int = 2
    S: int = 4

    @property
    def M(self) -> int:
        return len(self.theta_param)

    @property
    def D(self) -> int:
        return len(self.obs_index)

    @property
    def N(self) -> int:
        return self.theta_init.shape[0]

    @property
    def P(self) -> int:
        return self.M + (self.W - 1) * self.S

    def window_start(self, w: int) -> int:
        return (w * self.T) // self.W


def rigid_double_pendulum(N: int = 100, seed: int = 7000, T: int = 1000, W: int = 10,
                          theta_param=tuple(range(11))) -> Rigid2Workload:
    """All 11 true parameters ~ U over the middle half of the table's limits;
    recorded at 400 Hz (dt = 0.0025), T = 1000 steps (2.5 s), 10 windows;
    q0 ~ U(-pi/2, pi/2) at rest; both angles and both velocities observed with
    sigma 0.02 (velocities of the physical data come from finite differences);
    initial particles uniform in the limits of the estimated parameters."""
    rng = np.random.default_rng(seed)
    w = RIGID2_HI - RIGID2_LO
    p11 = rng.uniform(RIGID2_LO + 0.25 * w, RIGID2_HI - 0.25 * w)
    tp = np.asarray(theta_param, dtype=np.int32)
    lo, hi = RIGID2_LO[tp].copy(), RIGID2_HI[tp].copy()
    q0 = rng.uniform(-math.pi / 2, math.pi / 2, size=2)
    D = 4
    noise = rng.standard_normal((T, D))
    theta_init = rng.uniform(lo, hi, size=(N, len(tp)))
    return Rigid2Workload(name="rigid_double_pendulum", p11=p11, theta_param=tp, theta_true=p11[tp].copy(), lo=lo,
                          hi=hi, dt=0.0025, T=T, W=W, obs_index=np.arange(4, dtype=np.int32), sigma_obs=0.02,
                          sigma_def=SIGMA_DEF, s0=np.concatenate([q0, np.zeros(2)]), noise=noise,
                          theta_init=theta_init, seed=seed)


def serving_mix(n_jobs: int, seed: int = 5000, armbox_fraction: float = 0.1, armbox_N: int = 512):
    """Jobs of the serving workload: uneven chain problems, with a fraction of
    arm-shaking-a-box jobs at armbox_N particles (T = 2000, W = 40)."""
    rng = np.random.default_rng(seed)
    chains = batched_problems(n_jobs=n_jobs, seed=seed)
    out = []
    for j in range(n_jobs):
        if rng.uniform() < armbox_fraction:
            out.append(arm_box(N=armbox_N, seed=seed + 7919 * (j + 1)))
        else:
            out.append(chains[j])
    return out
