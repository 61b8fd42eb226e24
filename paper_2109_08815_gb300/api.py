"""Thin Python binding of libpds (include/pds.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; PyTorch only
supplies device memory and streams.  If ``libpds.so`` is missing or no CUDA
device is present, the calls raise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpds.so")

PDS_SYSTEM_PLANAR_CHAIN = 1
PARAM_MASS, PARAM_LENGTH, PARAM_DAMPING = 0, 1, 2
OPT_CHECKPOINT_STRIDE, OPT_FAST_MATH, OPT_MEDIAN_FULL_PASSES, OPT_PHI_CUDA_CORES, OPT_MEDIAN_CUDA_CORES = 1, 2, 3, 4, 5
OPT_WAIT_LIMIT = 6
OPT_GRAPH = 7
OPT_UNITS_PER_THREAD = 8
ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NONFINITE, ERR_TIMEOUT, ERR_BUDGET, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6, -7
COMBINE_SUM, COMBINE_PRODUCT = 0, 1
JOB_QUEUED, JOB_ACTIVE, JOB_DONE = 0, 1, 2
GATE_NONE, GATE_MMD2, GATE_KNN_KL = 0, 1, 2

_lib = None
_lock = threading.Lock()

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_fp = ctypes.POINTER(ctypes.c_float)


class _SystemDesc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("n_links", ctypes.c_int),
        ("mass", _dp),
        ("length", _dp),
        ("damping", _dp),
        ("gravity", ctypes.c_double),
        ("n_theta", ctypes.c_int),
        ("theta_kind", _ip),
        ("theta_link", _ip),
    ]


class _Rigid2Desc(ctypes.Structure):
    _fields_ = [
        ("param", ctypes.c_double * 11),
        ("gravity", ctypes.c_double),
        ("n_theta", ctypes.c_int),
        ("theta_param", _ip),
    ]


class _ArmBoxDesc(ctypes.Structure):
    _fields_ = [
        ("n_arm", ctypes.c_int),
        ("arm_len", _dp),
        ("amp", _dp),
        ("freq", _dp),
        ("phase", _dp),
        ("box_mass", ctypes.c_double),
        ("box_side", ctypes.c_double),
        ("box_com_depth", ctypes.c_double),
        ("weight_mass", ctypes.c_double * 2),
        ("weight_depth", ctypes.c_double),
        ("gravity", ctypes.c_double),
        ("damping", ctypes.c_double),
    ]


EXPORTS = {
    "pds_problem_create": ([ctypes.POINTER(_SystemDesc), ctypes.c_double, ctypes.c_int, ctypes.c_int, _fp,
                            ctypes.c_int, _ip, ctypes.c_double, ctypes.c_double, _fp, _fp, _fp, ctypes.c_double,
                            _vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "pds_problem_create_armbox": ([ctypes.POINTER(_ArmBoxDesc), ctypes.c_double, ctypes.c_int, ctypes.c_int, _fp,
                                   ctypes.c_int, _ip, ctypes.c_double, ctypes.c_double, _fp, _fp, _fp,
                                   ctypes.c_double, _vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "pds_problem_create_rigid2": ([ctypes.POINTER(_Rigid2Desc), ctypes.c_double, ctypes.c_int, ctypes.c_int, _fp,
                                   ctypes.c_int, _ip, ctypes.c_double, ctypes.c_double, _fp, _fp, _fp,
                                   ctypes.c_double, _vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "pds_problem_destroy": ([_vp], ctypes.c_int),
    "pds_problem_layout": ([_vp, _ip, _ip, _ip], ctypes.c_int),
    "pds_problem_set_checkpoint_stride": ([_vp, ctypes.c_int], ctypes.c_int),
    "pds_problem_reserve": ([_vp, ctypes.c_int], ctypes.c_int),
    "pds_problem_set_option": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "pds_problem_set_csvgd": ([_vp, ctypes.c_int, ctypes.c_double], ctypes.c_int),
    "pds_problem_set_trajectories": ([_vp, ctypes.c_int, _fp, _fp, ctypes.c_int], ctypes.c_int),
    "pds_knn_kl": ([_vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                    ctypes.POINTER(ctypes.c_double), _vp], ctypes.c_int),
    "pds_mmd2": ([_vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                  ctypes.POINTER(ctypes.c_double), _vp], ctypes.c_int),
    "pds_problem_get_option": ([_vp, ctypes.c_int, _ip], ctypes.c_int),
    "pds_problem_autotune": ([_vp, _vp, ctypes.c_int, _ip], ctypes.c_int),
    "pds_loglik_grad": ([_vp, _vp, ctypes.c_int, _vp, _vp, _vp], ctypes.c_int),
    "pds_simulate": ([_vp, _vp, ctypes.c_int, _vp], ctypes.c_int),
    "pds_svgd_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, _fp, _fp, ctypes.c_double, ctypes.c_double,
                         ctypes.c_double, ctypes.c_double, ctypes.c_int, _vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "pds_svgd_destroy": ([_vp], ctypes.c_int),
    "pds_svgd_step": ([_vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "pds_svgd_reset": ([_vp], ctypes.c_int),
    "pds_svgd_status": ([_vp], ctypes.c_int),
    "pds_svgd_set_option": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "pds_svgd_set_csvgd": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "pds_iterate": ([_vp, _vp, _vp, ctypes.c_int, _vp], ctypes.c_int),
    "pds_iterate_host": ([_vp, _vp, _vp, ctypes.c_int, _vp], ctypes.c_int),
    "pds_batch_create": ([ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                          ctypes.POINTER(_vp), _vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "pds_batch_destroy": ([_vp], ctypes.c_int),
    "pds_batch_autotune": ([_vp, ctypes.c_int, _ip], ctypes.c_int),
    "pds_batch_iterate": ([_vp, ctypes.c_int], ctypes.c_int),
    "pds_batch_info": ([_vp, _ip, _ip], ctypes.c_int),
    "pds_server_create": ([ctypes.c_size_t, ctypes.c_int, _vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "pds_server_destroy": ([_vp], ctypes.c_int),
    "pds_server_set_rollout_options": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "pds_server_submit": ([_vp, ctypes.POINTER(_SystemDesc), ctypes.c_double, ctypes.c_int, ctypes.c_int, _fp,
                           ctypes.c_int, _ip, ctypes.c_double, ctypes.c_double, _fp, _fp, _fp, ctypes.c_double,
                           ctypes.c_int, _fp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)],
                          ctypes.c_int),
    "pds_server_submit_rigid2": ([_vp, ctypes.POINTER(_Rigid2Desc), ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  _fp, ctypes.c_int, _ip, ctypes.c_double, ctypes.c_double, _fp, _fp, _fp,
                                  ctypes.c_double, ctypes.c_int, _fp, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    "pds_server_submit_armbox": ([_vp, ctypes.POINTER(_ArmBoxDesc), ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                  _fp, ctypes.c_int, _ip, ctypes.c_double, ctypes.c_double, _fp, _fp, _fp,
                                  ctypes.c_double, ctypes.c_int, _fp, ctypes.c_double, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    "pds_server_tick": ([_vp, _ip, _ip], ctypes.c_int),
    "pds_server_status": ([_vp, ctypes.c_longlong, _ip, _ip], ctypes.c_int),
    "pds_server_result": ([_vp, ctypes.c_longlong, _fp, _fp], ctypes.c_int),
    "pds_server_cancel": ([_vp, ctypes.c_longlong], ctypes.c_int),
    "pds_server_set_gate": ([_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double], ctypes.c_int),
    "pds_server_job_gate": ([_vp, ctypes.c_longlong, _ip, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "pds_server_stats": ([_vp, _ip, _ip, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "pds_sobol_box": ([_vp, ctypes.c_int, ctypes.c_int, _fp, _fp, ctypes.c_longlong, _vp], ctypes.c_int),
    "pds_sgld_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, _fp, _fp, ctypes.c_double, ctypes.c_double,
                         ctypes.c_double, ctypes.c_ulonglong, ctypes.c_int, _vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "pds_sgld_destroy": ([_vp], ctypes.c_int),
    "pds_sgld_reset": ([_vp], ctypes.c_int),
    "pds_sgld_step": ([_vp, _vp, _vp, _fp], ctypes.c_int),
    "pds_bandwidth_noalloc": ([_vp, ctypes.c_int, ctypes.c_int, _fp, _fp, _vp, _vp], ctypes.c_int),
    "pds_last_launch_count": ([], ctypes.c_int),
    "pds_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "pds_last_error": ([], ctypes.c_char_p),
}


class PdsError(RuntimeError):
    """A failed call; ``code`` is its PDS_ERR_* status (0 when the binding
    itself refused the call)."""

    def __init__(self, msg: str, code: int = 0):
        super().__init__(msg)
        self.code = code


def lib():
    """Load libpds.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise PdsError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in EXPORTS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        L = lib()
        raise PdsError(f"{what}: {L.pds_strerror(rc).decode()} ({rc}): {L.pds_last_error().decode()}", rc)


def last_launch_count() -> int:
    return int(lib().pds_last_launch_count())


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _need_cuda(t: torch.Tensor, dtype, name):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise PdsError(f"{name} must be a contiguous CUDA tensor of {dtype}")


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream), stream


class Problem:
    """A multiple-shooting inference problem (pds_problem_create).

    Arguments mirror :c:func:`pds_problem_create`; host arrays are numpy.
    ``obs`` is [T][D] with row t-1 = x_t.
    """

    def __init__(self, *, mass, length, damping, theta_kind, theta_link, dt, T, W, obs, obs_index, sigma_obs,
                 sigma_def, s0, lo, hi, g=9.81, c_lim=1e4, stream=None, checkpoint_stride=None, fast_math=None):
        L = lib()
        self._keep = []

        def d(x):
            a = np.ascontiguousarray(x, dtype=np.float64)
            self._keep.append(a)
            return a.ctypes.data_as(_dp)

        def i(x):
            a = np.ascontiguousarray(x, dtype=np.int32)
            self._keep.append(a)
            return a.ctypes.data_as(_ip)

        def f(x):
            a = np.ascontiguousarray(x, dtype=np.float32)
            self._keep.append(a)
            return a.ctypes.data_as(_fp)

        n = len(mass)
        obs = np.ascontiguousarray(obs, dtype=np.float32)
        self.T, self.W, self.n = int(T), int(W), n
        sysd = _SystemDesc(kind=PDS_SYSTEM_PLANAR_CHAIN, n_links=n, mass=d(mass), length=d(length),
                           damping=d(damping), gravity=float(g), n_theta=len(theta_kind), theta_kind=i(theta_kind),
                           theta_link=i(theta_link))
        self._stream_h, self.stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        _check(L.pds_problem_create(ctypes.byref(sysd), float(dt), self.T, self.W, f(obs), obs.shape[1],
                                    i(obs_index), float(sigma_obs), float(sigma_def), f(s0), f(lo), f(hi),
                                    float(c_lim), self._stream_h, ctypes.byref(h)), "pds_problem_create")
        self._h = h
        self._keep = []
        M, S, P = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(L.pds_problem_layout(h, ctypes.byref(M), ctypes.byref(S), ctypes.byref(P)), "pds_problem_layout")
        self.M, self.S, self.P = M.value, S.value, P.value
        if checkpoint_stride is not None:
            self.set_checkpoint_stride(checkpoint_stride)
        if fast_math is not None:
            self.set_option(OPT_FAST_MATH, int(bool(fast_math)))

    @classmethod
    def armbox(cls, wl, obs, stream=None, checkpoint_stride=None, fast_math=None):
        """Arm-and-box problem (pds_problem_create_armbox) from an ArmBoxWorkload."""
        self = cls.__new__(cls)
        L = lib()
        keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (wl.arm_len, wl.amp, wl.freq, wl.phase)]
        d = _ArmBoxDesc(n_arm=len(keep[0]), arm_len=keep[0].ctypes.data_as(_dp), amp=keep[1].ctypes.data_as(_dp),
                        freq=keep[2].ctypes.data_as(_dp), phase=keep[3].ctypes.data_as(_dp),
                        box_mass=wl.box_mass, box_side=wl.box_side, box_com_depth=wl.box_com_depth,
                        weight_mass=(ctypes.c_double * 2)(*wl.weight_mass), weight_depth=wl.weight_depth,
                        gravity=wl.g, damping=wl.box_damping)
        f = [np.ascontiguousarray(x, dtype=np.float32) for x in (obs, wl.s0, wl.lo, wl.hi)]
        oi = np.ascontiguousarray(wl.obs_index, dtype=np.int32)
        self._stream_h, self.stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        _check(L.pds_problem_create_armbox(ctypes.byref(d), float(wl.dt), int(wl.T), int(wl.W),
                                           f[0].ctypes.data_as(_fp), f[0].shape[1], oi.ctypes.data_as(_ip),
                                           float(wl.sigma_obs), float(wl.sigma_def), f[1].ctypes.data_as(_fp),
                                           f[2].ctypes.data_as(_fp), f[3].ctypes.data_as(_fp), float(wl.c_lim),
                                           self._stream_h, ctypes.byref(h)), "pds_problem_create_armbox")
        self._h = h
        self._keep = []
        self.T, self.W, self.n = int(wl.T), int(wl.W), 2
        M, S, P = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(L.pds_problem_layout(h, ctypes.byref(M), ctypes.byref(S), ctypes.byref(P)), "pds_problem_layout")
        self.M, self.S, self.P = M.value, S.value, P.value
        if checkpoint_stride is not None:
            self.set_checkpoint_stride(checkpoint_stride)
        if fast_math is not None:
            self.set_option(OPT_FAST_MATH, int(bool(fast_math)))
        return self

    @classmethod
    def rigid2(cls, wl, obs, stream=None, checkpoint_stride=None, fast_math=None):
        """Rigid double pendulum problem (pds_problem_create_rigid2) from a Rigid2Workload."""
        self = cls.__new__(cls)
        L = lib()
        tp = np.ascontiguousarray(wl.theta_param, dtype=np.int32)
        d = _Rigid2Desc(gravity=float(wl.g), n_theta=int(tp.size), theta_param=tp.ctypes.data_as(_ip))
        for k in range(11):
            d.param[k] = float(wl.p11[k])
        f = [np.ascontiguousarray(x, dtype=np.float32) for x in (obs, wl.s0, wl.lo, wl.hi)]
        oi = np.ascontiguousarray(wl.obs_index, dtype=np.int32)
        self._stream_h, self.stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        _check(L.pds_problem_create_rigid2(ctypes.byref(d), float(wl.dt), int(wl.T), int(wl.W),
                                           f[0].ctypes.data_as(_fp), f[0].shape[1], oi.ctypes.data_as(_ip),
                                           float(wl.sigma_obs), float(wl.sigma_def), f[1].ctypes.data_as(_fp),
                                           f[2].ctypes.data_as(_fp), f[3].ctypes.data_as(_fp), float(wl.c_lim),
                                           self._stream_h, ctypes.byref(h)), "pds_problem_create_rigid2")
        self._h = h
        self._keep = []
        self.T, self.W, self.n = int(wl.T), int(wl.W), 2
        M, S, P = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(L.pds_problem_layout(h, ctypes.byref(M), ctypes.byref(S), ctypes.byref(P)), "pds_problem_layout")
        self.M, self.S, self.P = M.value, S.value, P.value
        if checkpoint_stride is not None:
            self.set_checkpoint_stride(checkpoint_stride)
        if fast_math is not None:
            self.set_option(OPT_FAST_MATH, int(bool(fast_math)))
        return self

    @classmethod
    def from_workload(cls, wl, obs, **kw):
        if hasattr(wl, "arm_len"):
            return cls.armbox(wl, obs, **kw)
        if hasattr(wl, "p11"):
            return cls.rigid2(wl, obs, **kw)
        return cls(mass=wl.mass, length=wl.length, damping=wl.damping, theta_kind=wl.theta_kind,
                   theta_link=wl.theta_link, dt=wl.dt, T=wl.T, W=wl.W, obs=obs, obs_index=wl.obs_index,
                   sigma_obs=wl.sigma_obs, sigma_def=wl.sigma_def, s0=wl.s0, lo=wl.lo, hi=wl.hi, g=wl.g,
                   c_lim=wl.c_lim, **kw)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.pds_problem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_checkpoint_stride(self, K: int):
        _check(lib().pds_problem_set_checkpoint_stride(self._h, int(K)), "pds_problem_set_checkpoint_stride")

    def reserve(self, N: int):
        _check(lib().pds_problem_reserve(self._h, int(N)), "pds_problem_reserve")

    def set_option(self, option: int, value: int):
        _check(lib().pds_problem_set_option(self._h, int(option), int(value)), "pds_problem_set_option")

    def get_option(self, option: int) -> int:
        v = ctypes.c_int()
        _check(lib().pds_problem_get_option(self._h, int(option), ctypes.byref(v)), "pds_problem_get_option")
        return v.value

    def autotune(self, X) -> dict:
        """pds_problem_autotune on device particles X [P][N]: sets the fastest
        (units per thread, K) and returns it with its time per call."""
        ch = (ctypes.c_int * 3)()
        _check(lib().pds_problem_autotune(self._h, _ptr(X), int(X.shape[1]), ch), "pds_problem_autotune")
        return {"units_per_thread": ch[0], "K": ch[1], "us_per_call": ch[2]}

    def set_csvgd(self, enable: bool = True, c: float = 1.0):
        """Constrained SVGD (pds_problem_set_csvgd): observation likelihood,
        MDMM constraints; the layout grows by W-1 + M multiplier rows and the
        gradient has P + M rows."""
        L = lib()
        _check(L.pds_problem_set_csvgd(self._h, int(bool(enable)), float(c)), "pds_problem_set_csvgd")
        M, S, P = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(L.pds_problem_layout(self._h, ctypes.byref(M), ctypes.byref(S), ctypes.byref(P)), "pds_problem_layout")
        self.M, self.S, self.P = M.value, S.value, P.value
        self.csvgd = bool(enable)

    def set_trajectories(self, obs, s0, combine: str = "sum"):
        """A set of R trajectories (pds_problem_set_trajectories): obs [R][T][D],
        s0 [R][S]; combine "sum" (equally weighted mixture) or "product"."""
        obs = np.ascontiguousarray(obs, dtype=np.float32)
        s0 = np.ascontiguousarray(s0, dtype=np.float32)
        R = obs.shape[0]
        assert obs.ndim == 3 and s0.shape == (R, self.S), (obs.shape, s0.shape)
        mode = {"sum": COMBINE_SUM, "product": COMBINE_PRODUCT}[combine]
        L = lib()
        _check(L.pds_problem_set_trajectories(self._h, R, obs.ctypes.data_as(_fp), s0.ctypes.data_as(_fp), mode),
               "pds_problem_set_trajectories")
        M, S, P = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(L.pds_problem_layout(self._h, ctypes.byref(M), ctypes.byref(S), ctypes.byref(P)), "pds_problem_layout")
        self.M, self.S, self.P = M.value, S.value, P.value
        self.R = R

    @property
    def grad_rows(self) -> int:
        return self.P + (self.M if getattr(self, "csvgd", False) else 0)

    def loglik_grad(self, particles: torch.Tensor, grad: bool = True, out=None):
        """log p and (optionally) d log p / d particles for particles [P][N]
        (in constrained mode: log p_obs and the [P + M][N] rows of
        pds_problem_set_csvgd)."""
        _need_cuda(particles, torch.float32, "particles")
        assert particles.dim() == 2 and particles.shape[0] == self.P, (particles.shape, self.P)
        N = particles.shape[1]
        if out is None:
            logp = torch.empty(N, device=particles.device, dtype=torch.float32)
            g = torch.empty((self.grad_rows, N), device=particles.device, dtype=torch.float32) if grad else None
            status = torch.empty(N, device=particles.device, dtype=torch.int32)
        else:
            logp, g, status = out
        _check(lib().pds_loglik_grad(self._h, _ptr(particles), N, _ptr(logp), _ptr(g), _ptr(status)),
               "pds_loglik_grad")
        return logp, g, status

    def simulate(self, theta: torch.Tensor) -> torch.Tensor:
        """f_sim for theta [M][N]; returns states [T+1][S][N]."""
        _need_cuda(theta, torch.float32, "theta")
        N = theta.shape[1]
        states = torch.empty((self.T + 1, self.S, N), device=theta.device, dtype=torch.float32)
        _check(lib().pds_simulate(self._h, _ptr(theta), N, _ptr(states)), "pds_simulate")
        return states


class Svgd:
    """SVGD + Adam state (pds_svgd_create)."""

    def __init__(self, N, M, P, lo, hi, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, clamp=True, stream=None,
                 fast_math=False):
        L = lib()
        lo = np.ascontiguousarray(lo, dtype=np.float32)
        hi = np.ascontiguousarray(hi, dtype=np.float32)
        self._stream_h, self.stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        _check(L.pds_svgd_create(int(N), int(M), int(P), lo.ctypes.data_as(_fp), hi.ctypes.data_as(_fp), float(lr),
                                 float(beta1), float(beta2), float(eps), int(bool(clamp)), self._stream_h,
                                 ctypes.byref(h)), "pds_svgd_create")
        self._h = h
        self.N, self.M, self.P = int(N), int(M), int(P)
        if fast_math:
            _check(L.pds_svgd_set_option(h, OPT_FAST_MATH, 1), "pds_svgd_set_option")

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.pds_svgd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        _check(lib().pds_svgd_reset(self._h), "pds_svgd_reset")

    def status(self) -> int:
        """pds_svgd_status: synchronise the state's stream and return (and
        clear) what the device reported for the steps run so far: 0,
        ERR_TIMEOUT or ERR_NONFINITE."""
        return int(lib().pds_svgd_status(self._h))

    def set_option(self, option: int, value: int):
        _check(lib().pds_svgd_set_option(self._h, int(option), int(value)), "pds_svgd_set_option")

    def set_csvgd(self, n_def: int, enable: bool = True):
        """Constrained SVGD update (pds_svgd_set_csvgd) with n_def defect multipliers."""
        _check(lib().pds_svgd_set_csvgd(self._h, int(bool(enable)), int(n_def)), "pds_svgd_set_csvgd")

    def step(self, particles: torch.Tensor, grad: torch.Tensor, return_phi: bool = False):
        """In-place update of particles [P][N]; returns (bandwidth tensor, phi or None)."""
        _need_cuda(particles, torch.float32, "particles")
        _need_cuda(grad, torch.float32, "grad")
        bw = torch.empty(1, device=particles.device, dtype=torch.float32)
        phi = torch.empty((self.M, self.N), device=particles.device, dtype=torch.float32) if return_phi else None
        _check(lib().pds_svgd_step(self._h, _ptr(particles), _ptr(grad), _ptr(bw), _ptr(phi)), "pds_svgd_step")
        return bw, phi


def sobol_box(theta: torch.Tensor, lo, hi, skip: int = 0, stream=None) -> torch.Tensor:
    """Fill theta [M][N] (a contiguous CUDA float32 tensor, e.g. the first M
    rows of a particle array) with Sobol points scaled to the box
    (pds_sobol_box); returns theta."""
    _need_cuda(theta, torch.float32, "theta")
    assert theta.dim() == 2
    M, N = theta.shape
    lo = np.ascontiguousarray(lo, dtype=np.float32).reshape(-1)
    hi = np.ascontiguousarray(hi, dtype=np.float32).reshape(-1)
    assert lo.size == M and hi.size == M
    h, _ = _stream_handle(stream)
    _check(lib().pds_sobol_box(_ptr(theta), int(N), int(M), lo.ctypes.data_as(_fp), hi.ctypes.data_as(_fp),
                               int(skip), h), "pds_sobol_box")
    return theta


class Sgld:
    """Stochastic gradient Langevin dynamics chains (pds_sgld_create): one
    independent chain per particle, step size a (b + t)^(-gamma), theta rows
    moved in unit-box coordinates."""

    def __init__(self, N, M, P, lo, hi, a=1e-4, b=1.0, gamma=0.55, seed=0, clamp=True, stream=None):
        L = lib()
        lo = np.ascontiguousarray(lo, dtype=np.float32).reshape(-1)
        hi = np.ascontiguousarray(hi, dtype=np.float32).reshape(-1)
        assert lo.size == M and hi.size == M
        self._stream_h, self.stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        _check(L.pds_sgld_create(int(N), int(M), int(P), lo.ctypes.data_as(_fp), hi.ctypes.data_as(_fp), float(a),
                                 float(b), float(gamma), int(seed) & (2 ** 64 - 1), int(bool(clamp)), self._stream_h,
                                 ctypes.byref(h)), "pds_sgld_create")
        self._h = h
        self.N, self.M, self.P = int(N), int(M), int(P)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.pds_sgld_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self):
        _check(lib().pds_sgld_reset(self._h), "pds_sgld_reset")

    def step(self, particles: torch.Tensor, grad: torch.Tensor) -> float:
        """In-place update of particles [P][N] with gradient [P][N]; returns eps_t."""
        _need_cuda(particles, torch.float32, "particles")
        _need_cuda(grad, torch.float32, "grad")
        assert tuple(particles.shape) == (self.P, self.N) and tuple(grad.shape) == (self.P, self.N)
        eps = ctypes.c_float()
        _check(lib().pds_sgld_step(self._h, _ptr(particles), _ptr(grad), ctypes.byref(eps)), "pds_sgld_step")
        return eps.value


def knn_kl(p: torch.Tensor, q: torch.Tensor, k: int = 3, stream=None) -> float:
    """KNN estimate of KL(P || Q) (pds_knn_kl) for sample sets p [d][n], q [d][m]."""
    _need_cuda(p, torch.float32, "p")
    _need_cuda(q, torch.float32, "q")
    assert p.dim() == 2 and q.dim() == 2 and p.shape[0] == q.shape[0]
    h, _ = _stream_handle(stream)
    out = ctypes.c_double()
    _check(lib().pds_knn_kl(_ptr(p), p.shape[1], _ptr(q), q.shape[1], p.shape[0], int(k), ctypes.byref(out), h),
           "pds_knn_kl")
    return out.value


def mmd2(x: torch.Tensor, y: torch.Tensor, h: float, stream=None) -> float:
    """Unbiased MMD^2 with the RBF kernel exp(-|x - y|^2 / h) (pds_mmd2); x [d][n], y [d][m]."""
    _need_cuda(x, torch.float32, "x")
    _need_cuda(y, torch.float32, "y")
    assert x.dim() == 2 and y.dim() == 2 and x.shape[0] == y.shape[0]
    sh, _ = _stream_handle(stream)
    out = ctypes.c_double()
    _check(lib().pds_mmd2(_ptr(x), x.shape[1], _ptr(y), y.shape[1], x.shape[0], float(h), ctypes.byref(out), sh),
           "pds_mmd2")
    return out.value


def iterate(problem: Problem, svgd: Svgd, particles: torch.Tensor, iters: int, logp: torch.Tensor | None = None):
    """Algorithm 1 on the device: iters x (log p + gradient, SVGD update)."""
    _need_cuda(particles, torch.float32, "particles")
    _check(lib().pds_iterate(problem.handle, svgd.handle, _ptr(particles), int(iters), _ptr(logp)), "pds_iterate")


def iterate_host(problem: Problem, svgd: Svgd, particles: np.ndarray, iters: int, logp: np.ndarray | None = None):
    """Algorithm 1 on host-resident float32 arrays (copies inside the call)."""
    assert particles.dtype == np.float32 and particles.flags.c_contiguous
    lp = None if logp is None else ctypes.c_void_p(logp.ctypes.data)
    _check(lib().pds_iterate_host(problem.handle, svgd.handle, ctypes.c_void_p(particles.ctypes.data), int(iters),
                                  lp), "pds_iterate_host")


class Batch:
    """Many problems iterated together (pds_batch_*): one persistent rollout
    launch per chain length plus per-problem SVGD branches, replayed from a
    captured CUDA graph."""

    def __init__(self, problems, svgds, particles, logp=None, stream=None):
        L = lib()
        n = len(problems)
        assert len(svgds) == n and len(particles) == n
        for x in particles:
            _need_cuda(x, torch.float32, "particles")
        self._problems, self._svgds, self._particles = list(problems), list(svgds), list(particles)
        self._logp = list(logp) if logp is not None else None
        arr = lambda xs: (_vp * n)(*[ctypes.c_void_p(x) for x in xs])  # noqa: E731
        ph = arr([p.handle.value for p in problems])
        sh = arr([s.handle.value for s in svgds])
        xh = arr([x.data_ptr() for x in particles])
        lh = arr([t.data_ptr() for t in logp]) if logp is not None else None
        self._stream_h, self.stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        _check(L.pds_batch_create(n, ph, sh, xh, lh, self._stream_h, ctypes.byref(h)), "pds_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.pds_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, allow_fast_math=True):
        """Returns [(links, K, fast_math, grid_blocks, units_per_thread)] per chain length."""
        ng, _ = self.info()
        ch = (ctypes.c_int * (5 * max(ng, 1)))()
        _check(lib().pds_batch_autotune(self._h, int(bool(allow_fast_math)), ch), "pds_batch_autotune")
        ng, _ = self.info()
        return [tuple(ch[5 * g:5 * g + 5]) for g in range(ng)]

    def iterate(self, iters=1):
        _check(lib().pds_batch_iterate(self._h, int(iters)), "pds_batch_iterate")

    def info(self):
        ng, lpi = ctypes.c_int(), ctypes.c_int()
        _check(lib().pds_batch_info(self._h, ctypes.byref(ng), ctypes.byref(lpi)), "pds_batch_info")
        return ng.value, lpi.value


class Server:
    """Serving loop with continuous batching (pds_server_*)."""

    def __init__(self, mem_budget_bytes: int, max_active: int = 256, stream=None, checkpoint_stride=None,
                 fast_math=None):
        L = lib()
        self._stream_h, self.stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        _check(L.pds_server_create(int(mem_budget_bytes), int(max_active), self._stream_h, ctypes.byref(h)),
               "pds_server_create")
        self._h = h
        if checkpoint_stride is not None or fast_math is not None:
            _check(L.pds_server_set_rollout_options(h, int(checkpoint_stride or 1), int(1 if fast_math is None
                                                                                         else bool(fast_math))),
                   "pds_server_set_rollout_options")
        self._shapes = {}

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.pds_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, wl, obs, particles: np.ndarray, iterations: int) -> int:
        """Submit a workload-shaped job; particles [N][P] (host)."""
        keep = []

        def d(x):
            a = np.ascontiguousarray(x, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data_as(_dp)

        def i(x):
            a = np.ascontiguousarray(x, dtype=np.int32)
            keep.append(a)
            return a.ctypes.data_as(_ip)

        def f(x):
            a = np.ascontiguousarray(x, dtype=np.float32)
            keep.append(a)
            return a.ctypes.data_as(_fp)

        obs = np.ascontiguousarray(obs, dtype=np.float32)
        x = np.ascontiguousarray(np.asarray(particles).T, dtype=np.float32)  # [P][N]
        jid = ctypes.c_longlong()
        if hasattr(wl, "p11"):
            rd = _Rigid2Desc(gravity=float(wl.g), n_theta=len(wl.theta_param), theta_param=i(wl.theta_param))
            for k in range(11):
                rd.param[k] = float(wl.p11[k])
            _check(lib().pds_server_submit_rigid2(self._h, ctypes.byref(rd), float(wl.dt), int(wl.T), int(wl.W),
                                                  f(obs), obs.shape[1], i(wl.obs_index), float(wl.sigma_obs),
                                                  float(wl.sigma_def), f(wl.s0), f(wl.lo), f(wl.hi),
                                                  float(wl.c_lim), x.shape[1], f(x), float(wl.lr), int(iterations),
                                                  ctypes.byref(jid)), "pds_server_submit_rigid2")
        elif hasattr(wl, "arm_len"):
            ad = _ArmBoxDesc(n_arm=len(wl.arm_len), arm_len=d(wl.arm_len), amp=d(wl.amp), freq=d(wl.freq),
                             phase=d(wl.phase), box_mass=wl.box_mass, box_side=wl.box_side,
                             box_com_depth=wl.box_com_depth, weight_mass=(ctypes.c_double * 2)(*wl.weight_mass),
                             weight_depth=wl.weight_depth, gravity=wl.g, damping=wl.box_damping)
            _check(lib().pds_server_submit_armbox(self._h, ctypes.byref(ad), float(wl.dt), int(wl.T), int(wl.W),
                                                  f(obs), obs.shape[1], i(wl.obs_index), float(wl.sigma_obs),
                                                  float(wl.sigma_def), f(wl.s0), f(wl.lo), f(wl.hi),
                                                  float(wl.c_lim), x.shape[1], f(x), float(wl.lr), int(iterations),
                                                  ctypes.byref(jid)), "pds_server_submit_armbox")
        else:
            sysd = _SystemDesc(kind=PDS_SYSTEM_PLANAR_CHAIN, n_links=wl.n, mass=d(wl.mass), length=d(wl.length),
                               damping=d(wl.damping), gravity=float(wl.g), n_theta=wl.M,
                               theta_kind=i(wl.theta_kind), theta_link=i(wl.theta_link))
            _check(lib().pds_server_submit(self._h, ctypes.byref(sysd), float(wl.dt), int(wl.T), int(wl.W),
                                           f(obs), obs.shape[1], i(wl.obs_index), float(wl.sigma_obs),
                                           float(wl.sigma_def), f(wl.s0), f(wl.lo), f(wl.hi), float(wl.c_lim),
                                           x.shape[1], f(x), float(wl.lr), int(iterations), ctypes.byref(jid)),
                   "pds_server_submit")
        self._shapes[jid.value] = (x.shape[0], x.shape[1])
        return jid.value

    def tick(self):
        a, r = ctypes.c_int(), ctypes.c_int()
        _check(lib().pds_server_tick(self._h, ctypes.byref(a), ctypes.byref(r)), "pds_server_tick")
        return a.value, r.value

    def status(self, job_id):
        st, it = ctypes.c_int(), ctypes.c_int()
        _check(lib().pds_server_status(self._h, ctypes.c_longlong(job_id), ctypes.byref(st), ctypes.byref(it)),
               "pds_server_status")
        return st.value, it.value

    def result(self, job_id):
        """(particles [N][P], logp [N]) of a finished job; forgets the job."""
        P, N = self._shapes.pop(job_id)
        x = np.empty((P, N), np.float32)
        lp = np.empty(N, np.float32)
        _check(lib().pds_server_result(self._h, ctypes.c_longlong(job_id), x.ctypes.data_as(_fp),
                                       lp.ctypes.data_as(_fp)), "pds_server_result")
        return x.T.copy(), lp

    def cancel(self, job_id):
        _check(lib().pds_server_cancel(self._h, ctypes.c_longlong(job_id)), "pds_server_cancel")
        self._shapes.pop(job_id, None)

    def set_gate(self, metric: int, every: int, threshold: float, h: float = 0.1):
        """Convergence gate (pds_server_set_gate): retire a job once the metric
        between successive theta snapshots is <= threshold."""
        _check(lib().pds_server_set_gate(self._h, int(metric), int(every), float(threshold), float(h)),
               "pds_server_set_gate")

    def gate(self, job_id):
        """(number of gate evaluations, last value) of a job."""
        c, v = ctypes.c_int(), ctypes.c_double()
        _check(lib().pds_server_job_gate(self._h, ctypes.c_longlong(job_id), ctypes.byref(c), ctypes.byref(v)),
               "pds_server_job_gate")
        return c.value, v.value

    def stats(self):
        q, a, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
        _check(lib().pds_server_stats(self._h, ctypes.byref(q), ctypes.byref(a), ctypes.byref(b)),
               "pds_server_stats")
        return q.value, a.value, b.value


class LogLik(torch.autograd.Function):
    """log p(particles) as a differentiable torch op: the backward pass uses
    the hand-written adjoint computed by the same kernel launch."""

    @staticmethod
    def forward(ctx, particles, problem):
        logp, g, _ = problem.loglik_grad(particles.detach().contiguous(), grad=True)
        ctx.save_for_backward(g)
        return logp

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return g * grad_out[None, :], None


def loglik(particles: torch.Tensor, problem: Problem) -> torch.Tensor:
    return LogLik.apply(particles, problem)


def bandwidth_noalloc(theta: torch.Tensor, lo, hi, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Median-heuristic bandwidth of theta [M][N] through the entry point that
    allocates no device memory (for callers that cannot call cudaMalloc)."""
    _need_cuda(theta, torch.float32, "theta")
    M, N = theta.shape
    lo = np.ascontiguousarray(lo, dtype=np.float32)
    hi = np.ascontiguousarray(hi, dtype=np.float32)
    if out is None:
        out = torch.empty(1, device=theta.device, dtype=torch.float32)
    h, _ = _stream_handle(stream)
    _check(lib().pds_bandwidth_noalloc(_ptr(theta), int(N), int(M), lo.ctypes.data_as(_fp), hi.ctypes.data_as(_fp),
                                       _ptr(out), h), "pds_bandwidth_noalloc")
    return out
