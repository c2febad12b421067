"""ctypes wrapper of the FP64 Shield-MPPI oracle (smppi_oracle.cpp).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of bench.py may use it; the product path never does.  See smppi_oracle.cpp for
the passages of arXiv 2302.11719 each routine follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smppi_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (IEEE double, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class OrcParams(C.Structure):
    _fields_ = [
        ("m", C.c_double), ("Iz", C.c_double), ("lf", C.c_double), ("lr", C.c_double),
        ("B", C.c_double), ("Ct", C.c_double), ("g", C.c_double), ("fx_gain", C.c_double),
        ("dt", C.c_double),
        ("sigma", C.c_double * 2),
        ("lam", C.c_double), ("gamma", C.c_double),
        ("K", C.c_int), ("T", C.c_int), ("N_r", C.c_int),
        ("alpha", C.c_double), ("C_cbf", C.c_double),
        ("q_v", C.c_double), ("v_target", C.c_double), ("q_d", C.c_double), ("C_obs", C.c_double),
        ("u_min", C.c_double * 2), ("u_max", C.c_double * 2),
        ("half_width", C.c_double),
        ("dist_sigma", C.c_double * 2),
        ("ls_s0", C.c_double), ("ls_c", C.c_double),
        ("ls_max_halvings", C.c_int),
        ("n_track", C.c_int),
        ("track_xy", C.POINTER(C.c_float)),
        ("seed", C.c_uint64),
        ("state_kind", C.c_int),
        ("kappa", C.POINTER(C.c_double)),
        ("track_len", C.c_double),
    ]


_dp = C.POINTER(C.c_double)
_PP = C.POINTER(OrcParams)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        u32p, u64p = C.POINTER(C.c_uint32), C.POINTER(C.c_uint64)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_philox4x64_10.argtypes = [u64p, u64p, u64p]
        L.orc_uniform.argtypes = [C.c_uint32]; L.orc_uniform.restype = C.c_double
        L.orc_box_muller.argtypes = [C.c_uint32, C.c_uint32, _dp]
        L.orc_normal_pair.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                      C.c_uint32, C.c_uint32, _dp]
        L.orc_noise.argtypes = [_PP, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, _dp]
        L.orc_disturbance.argtypes = [_PP, C.c_uint32, C.c_uint32, _dp]
        L.orc_noise_block.argtypes = [_PP, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, C.c_int,
                                      _dp]
        L.orc_seg_dist2.argtypes = [_PP, C.c_int, C.c_double, C.c_double]
        L.orc_seg_dist2.restype = C.c_double
        L.orc_kappa_at.argtypes = [_PP, C.c_double]
        L.orc_kappa_at.restype = C.c_double
        L.orc_track_nearest.argtypes = [_PP, C.c_double, C.c_double, _dp]
        L.orc_track_nearest.restype = C.c_int
        L.orc_track_follow.argtypes = [_PP, C.c_int, C.c_double, C.c_double, _dp]
        L.orc_track_follow.restype = C.c_int
        L.orc_h.argtypes = [_PP, C.c_double]; L.orc_h.restype = C.c_double
        L.orc_q.argtypes = [_PP, _dp, C.c_double]; L.orc_q.restype = C.c_double
        L.orc_cbf_penalty.argtypes = [_PP, C.c_double, C.c_double]
        L.orc_cbf_penalty.restype = C.c_double
        L.orc_deriv.argtypes = [_PP, _dp, _dp, _dp]
        L.orc_step.argtypes = [_PP, _dp, _dp, _dp]
        L.orc_rollout.argtypes = [_PP, _dp, _dp, C.c_uint32, C.c_uint32, C.c_uint32, C.c_int,
                                  _dp, _dp]
        L.orc_rollout.restype = C.c_double
        L.orc_update.argtypes = [_PP, _dp, _dp, C.c_uint32, C.c_uint32, _dp, _dp]
        L.orc_mppi_step.argtypes = [_PP, _dp, _dp, C.c_uint32, C.c_uint32, _dp, _dp, C.c_int]
        L.orc_partial.argtypes = [_PP, _dp, C.c_uint32, C.c_uint32, C.c_int, C.c_int, _dp]
        L.orc_merge.argtypes = [_PP, C.c_int, _dp, _dp, _dp]
        L.orc_cost.argtypes = [_PP, _dp, _dp, C.c_int, C.c_double, C.c_double]
        L.orc_cost.restype = C.c_double
        L.orc_merit.argtypes = [_PP, _dp, _dp]; L.orc_merit.restype = C.c_double
        L.orc_cost_grad.argtypes = [_PP, _dp, _dp, C.c_int, C.c_double, C.c_double, _dp]
        L.orc_cost_grad.restype = C.c_double
        L.orc_repair.argtypes = [_PP, _dp, _dp, C.c_int, C.c_int, C.c_double, _dp,
                                 C.POINTER(C.c_int)]
        L.orc_repair.restype = C.c_int
        L.orc_bfgs_update.argtypes = [C.c_int, _dp, _dp, _dp]
        L.orc_bfgs_quadratic.argtypes = [C.c_int, _dp, _dp, _dp, _dp, _dp, C.c_int, C.c_double,
                                         C.c_double, C.c_int, _dp, C.POINTER(C.c_int)]
        L.orc_bfgs_quadratic.restype = C.c_int
        L.orc_apply.argtypes = [_PP, _dp, _dp, C.c_uint32, C.c_uint32, _dp]
        L.orc_curvature_table.argtypes = [_PP, _dp, _dp]
        L.orc_shift.argtypes = [_PP, _dp, _dp]
        L.orc_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _f32(v) -> float:
    """Parameter values are the float32 ones the GPU path uses."""
    return float(np.float32(v))


class Model:
    """Parameters + centreline of one problem, as the oracle sees them."""

    def __init__(self, params: dict, track: np.ndarray):
        self.track = np.ascontiguousarray(track, dtype=np.float32)
        p = OrcParams()
        for name in ("m", "Iz", "lf", "lr", "B", "Ct", "g", "fx_gain", "dt", "gamma", "alpha",
                     "C_cbf", "q_v", "v_target", "q_d", "C_obs", "half_width", "ls_s0"):
            setattr(p, name, _f32(params[name]))
        p.lam = _f32(params["lam"])
        p.ls_c = float(params["ls_c"])
        for name in ("sigma", "u_min", "u_max", "dist_sigma"):
            arr = getattr(p, name)
            arr[0], arr[1] = _f32(params[name][0]), _f32(params[name][1])
        p.K, p.T, p.N_r = int(params["K"]), int(params["T"]), int(params["N_r"])
        p.ls_max_halvings = int(params["ls_max_halvings"])
        p.n_track = int(self.track.shape[0])
        p.track_xy = self.track.ctypes.data_as(C.POINTER(C.c_float))
        p.seed = int(params["seed"])
        p.state_kind = int(params.get("state_kind", 0))
        self.p = p
        self.ptr = C.pointer(self.p)
        self.kappa = None
        if p.state_kind == 1:
            self.kappa = np.zeros(p.n_track)
            L = C.c_double()
            lib().orc_curvature_table(self.ptr, self.kappa.ctypes.data_as(_dp), C.byref(L))
            p.kappa = self.kappa.ctypes.data_as(_dp)
            p.track_len = L.value

    @property
    def K(self):
        return self.p.K

    @property
    def T(self):
        return self.p.T

    def with_(self, **kw) -> "Model":
        """Copy with some fields changed (K, T, N_r, lam, gamma, sigma, ...)."""
        m = Model.__new__(Model)
        m.track = self.track
        m.p = OrcParams.from_buffer_copy(self.p)
        m.p.track_xy = self.track.ctypes.data_as(C.POINTER(C.c_float))
        m.kappa = self.kappa
        if self.kappa is not None:
            m.p.kappa = self.kappa.ctypes.data_as(_dp)
        for k, v in kw.items():
            if k in ("sigma", "u_min", "u_max", "dist_sigma"):
                arr = getattr(m.p, k)
                arr[0], arr[1] = _f32(v[0]), _f32(v[1])
            elif k in ("K", "T", "N_r", "ls_max_halvings", "seed"):
                setattr(m.p, k, int(v))
            else:
                setattr(m.p, k, _f32(v))
        m.ptr = C.pointer(m.p)
        return m


def _d(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        assert a.size == n, (a.size, n)
    return a, a.ctypes.data_as(_dp)


def philox4x32(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def philox4x64(ctr, key):
    c = (C.c_uint64 * 4)(*[int(x) for x in ctr])
    k = (C.c_uint64 * 2)(*[int(x) for x in key])
    o = (C.c_uint64 * 4)()
    lib().orc_philox4x64_10(c, k, o)
    return [int(x) for x in o]


def uniform(x: int) -> float:
    return lib().orc_uniform(int(x))


def box_muller(a: int, b: int):
    z = np.zeros(2)
    lib().orc_box_muller(int(a), int(b), z.ctypes.data_as(_dp))
    return z


def normal_pair(seed, it, instance, stream, k, t):
    z = np.zeros(2)
    lib().orc_normal_pair(int(seed), int(it), int(instance), int(stream), int(k), int(t),
                          z.ctypes.data_as(_dp))
    return z


def noise(m: Model, it, instance, k, t):
    e = np.zeros(2)
    lib().orc_noise(m.ptr, int(it), int(instance), int(k), int(t), e.ctypes.data_as(_dp))
    return e


def noise_block(m: Model, it, instance, ks, T=None):
    """eps for rollouts ks and steps 0..T-1: (len(ks), T, 2)."""
    T = m.T if T is None else T
    ks = list(ks)
    out = np.zeros((len(ks), T, 2))
    if ks and ks == list(range(ks[0], ks[0] + len(ks))):
        lib().orc_noise_block(m.ptr, int(it), int(instance), int(ks[0]), len(ks), int(T),
                              out.ctypes.data_as(_dp))
        return out
    for i, k in enumerate(ks):
        for t in range(T):
            out[i, t] = noise(m, it, instance, k, t)
    return out


def disturbance(m: Model, n, instance=0):
    w = np.zeros(6)
    lib().orc_disturbance(m.ptr, int(n), int(instance), w.ctypes.data_as(_dp))
    return w


def deriv(m: Model, x, u):
    x, xp = _d(x, 6); u, up = _d(u, 2)
    out = np.zeros(6)
    lib().orc_deriv(m.ptr, xp, up, out.ctypes.data_as(_dp))
    return out


def step(m: Model, x, u):
    x, xp = _d(x, 6); u, up = _d(u, 2)
    out = np.zeros(6)
    lib().orc_step(m.ptr, xp, up, out.ctypes.data_as(_dp))
    return out


def seg_dist2(m: Model, i, X, Y):
    return lib().orc_seg_dist2(m.ptr, int(i), float(X), float(Y))


def kappa_at(m: Model, s):
    """kappa(s) of the curvilinear model (state_kind 1): the curvature samples
    interpolated linearly in arc length, s taken modulo the track length."""
    assert m.kappa is not None, "kappa(s) needs a curvilinear model (state_kind 1)"
    return lib().orc_kappa_at(m.ptr, float(s))


def track_nearest(m: Model, X, Y):
    d2 = C.c_double()
    s = lib().orc_track_nearest(m.ptr, float(X), float(Y), C.byref(d2))
    return s, d2.value


def track_follow(m: Model, seg, X, Y):
    d2 = C.c_double()
    s = lib().orc_track_follow(m.ptr, int(seg), float(X), float(Y), C.byref(d2))
    return s, d2.value


def h(m: Model, d2):
    return lib().orc_h(m.ptr, float(d2))


def q(m: Model, x, d2):
    x, xp = _d(x, 6)
    return lib().orc_q(m.ptr, xp, float(d2))


def cbf_penalty(m: Model, h_prev, h_now):
    return lib().orc_cbf_penalty(m.ptr, float(h_prev), float(h_now))


def rollout(m: Model, x0, V, k=0, it=0, instance=0, noisy=True):
    """(S~, traj (T+1, 6), eps (T, 2)) of rollout k."""
    x0, xp = _d(x0, 6); V, vp = _d(V, 2 * m.T)
    traj = np.zeros((m.T + 1, 6)); eps = np.zeros((m.T, 2))
    S = lib().orc_rollout(m.ptr, xp, vp, int(it), int(instance), int(k), int(bool(noisy)),
                          traj.ctypes.data_as(_dp), eps.ctypes.data_as(_dp))
    return S, traj, eps


def update(m: Model, S, V, it=0, instance=0):
    """(V+ (T, 2), normalised weights omega (K,)) from given costs S."""
    S, sp = _d(S, m.K); V, vp = _d(V, 2 * m.T)
    vplus = np.zeros((m.T, 2)); om = np.zeros(m.K)
    lib().orc_update(m.ptr, sp, vp, int(it), int(instance), vplus.ctypes.data_as(_dp),
                     om.ctypes.data_as(_dp))
    return vplus, om


def partial(m: Model, S_slice, k_lo, it=0, instance=0):
    """(m_g, eta_g, A_g) of rollouts k_lo .. k_lo + len(S_slice) - 1 from their
    costs: a float64 array of 2T + 2 values."""
    S, sp = _d(S_slice)
    out = np.zeros(2 * m.T + 2)
    lib().orc_partial(m.ptr, sp, int(it), int(instance), int(k_lo), int(k_lo + S.size),
                      out.ctypes.data_as(_dp))
    return out


def merge(m: Model, parts, V):
    """V+ (T, 2) from slice partials (n_parts, 2T + 2)."""
    P = np.ascontiguousarray(parts, np.float64).reshape(-1, 2 * m.T + 2)
    V, vp = _d(V, 2 * m.T)
    out = np.zeros((m.T, 2))
    lib().orc_merge(m.ptr, P.shape[0], P.ctypes.data_as(_dp), vp, out.ctypes.data_as(_dp))
    return out


def mppi_step(m: Model, x0, V, it=0, instance=0, nthreads=1):
    """(S (K,), V+ (T, 2)) of one MPPI iteration."""
    x0, xp = _d(x0, 6); V, vp = _d(V, 2 * m.T)
    S = np.zeros(m.K); vplus = np.zeros((m.T, 2))
    lib().orc_mppi_step(m.ptr, xp, vp, int(it), int(instance), S.ctypes.data_as(_dp),
                        vplus.ctypes.data_as(_dp), int(nthreads))
    return S, vplus


def cost(m: Model, x0, V, N=None, w_run=0.0, w_cbf=1.0):
    N = m.T if N is None else N
    x0, xp = _d(x0, 6); V, vp = _d(V, 2 * m.T)
    return lib().orc_cost(m.ptr, xp, vp, int(N), float(w_run), float(w_cbf))


def merit(m: Model, x0, V):
    x0, xp = _d(x0, 6); V, vp = _d(V, 2 * m.T)
    return lib().orc_merit(m.ptr, xp, vp)


def cost_grad(m: Model, x0, V, N=None, w_run=0.0, w_cbf=1.0):
    """(J, dJ/dV (T, 2)) by forward-mode dual numbers."""
    N = m.T if N is None else N
    x0, xp = _d(x0, 6); V, vp = _d(V, 2 * m.T)
    g = np.zeros((m.T, 2))
    J = lib().orc_cost_grad(m.ptr, xp, vp, int(N), float(w_run), float(w_cbf),
                            g.ctypes.data_as(_dp))
    return J, g


def repair(m: Model, x0, V, n_iters, mode=1, delta=0.0):
    """(V_safe (T, 2), merit (n_iters + 1,), status, iterations run).
    mode 0: fixed step, 1: projected gradient + Armijo, 2: BFGS."""
    x0, xp = _d(x0, 6)
    Vs = np.array(V, dtype=np.float64).reshape(m.T, 2).copy()
    mer = np.zeros(n_iters + 1)
    it = C.c_int()
    st = lib().orc_repair(m.ptr, xp, Vs.ctypes.data_as(_dp), int(n_iters), int(mode),
                          float(delta), mer.ctypes.data_as(_dp), C.byref(it))
    return Vs, mer, st, it.value


def bfgs_update(H, s, y):
    """The inverse BFGS update (I - rho s y') H (I - rho y s') + rho s s' (a new array)."""
    n = len(s)
    Hn = np.array(H, dtype=np.float64).reshape(n, n).copy()
    s = np.ascontiguousarray(s, np.float64); y = np.ascontiguousarray(y, np.float64)
    lib().orc_bfgs_update(n, Hn.ctypes.data_as(_dp), s.ctypes.data_as(_dp), y.ctypes.data_as(_dp))
    return Hn


def bfgs_quadratic(A, b, lo, hi, z0, n_iters, s0=0.1, c=1e-4, ls_max=20):
    """Box BFGS (the repair's mode-2 solver) on 1/2 z'Az - b'z:
    (z, f before each iteration and after the last, status, iterations run)."""
    n = len(b)
    A = np.ascontiguousarray(A, np.float64); b = np.ascontiguousarray(b, np.float64)
    lo = np.ascontiguousarray(lo, np.float64); hi = np.ascontiguousarray(hi, np.float64)
    z = np.array(z0, dtype=np.float64).copy()
    mer = np.zeros(n_iters + 1)
    it = C.c_int()
    st = lib().orc_bfgs_quadratic(n, A.ctypes.data_as(_dp), b.ctypes.data_as(_dp),
                                  lo.ctypes.data_as(_dp), hi.ctypes.data_as(_dp),
                                  z.ctypes.data_as(_dp), int(n_iters), float(s0), float(c),
                                  int(ls_max), mer.ctypes.data_as(_dp), C.byref(it))
    return z, mer, st, it.value


def apply(m: Model, x0, v0, n, instance=0):
    x0, xp = _d(x0, 6); v0, vp = _d(v0, 2)
    out = np.zeros(6)
    lib().orc_apply(m.ptr, xp, vp, int(n), int(instance), out.ctypes.data_as(_dp))
    return out


def shift(m: Model, Vplus):
    Vp, vp = _d(Vplus, 2 * m.T)
    out = np.zeros((m.T, 2))
    lib().orc_shift(m.ptr, vp, out.ctypes.data_as(_dp))
    return out


def curvature_table(m: Model):
    """(kappa samples at the n uniform arc-length stations, track length L)."""
    k = np.zeros(m.p.n_track)
    L = C.c_double()
    lib().orc_curvature_table(m.ptr, k.ctypes.data_as(_dp), C.byref(L))
    return k, L.value


def max_threads() -> int:
    return lib().orc_max_threads()
