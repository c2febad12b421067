"""Thin Python binding of libsmppi.so (include/smppi.h): argument marshalling only.

Every function here forwards to the C ABI entry point of the same name; all
computation runs in the library's CUDA kernels.  Tensors are torch CUDA
tensors (float32 unless stated, contiguous); PyTorch supplies device memory
and streams.  There is no CPU fallback: if the library is missing the import
of this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsmppi.so")

OK, ERR_ARG, ERR_CUDA, ERR_NUMERIC, ERR_TIMEOUT, ERR_STALLED, ERR_NOMEM = range(7)
DEV_NUMERIC, DEV_TIMEOUT, DEV_STALLED = 1, 2, 4
MAX_T, MAX_TRACK = 512, 2048


class SmppiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("smppi status %d: %s" % (status, msg))
        self.status = status


class Params(C.Structure):
    _fields_ = [
        ("m", C.c_float), ("Iz", C.c_float), ("lf", C.c_float), ("lr", C.c_float),
        ("B", C.c_float), ("Ct", C.c_float), ("g", C.c_float), ("fx_gain", C.c_float),
        ("dt", C.c_float),
        ("sigma", C.c_float * 2),
        ("lam", C.c_float), ("gamma", C.c_float),
        ("K", C.c_int), ("T", C.c_int), ("N_r", C.c_int),
        ("alpha", C.c_float), ("C_cbf", C.c_float),
        ("q_v", C.c_float), ("v_target", C.c_float), ("q_d", C.c_float), ("C_obs", C.c_float),
        ("u_min", C.c_float * 2), ("u_max", C.c_float * 2),
        ("half_width", C.c_float),
        ("dist_sigma", C.c_float * 2),
        ("ls_s0", C.c_float), ("ls_c", C.c_float),
        ("ls_max_halvings", C.c_int),
        ("checkpoint", C.c_int),
        ("max_seq", C.c_int),
        ("n_track", C.c_int),
        ("track_xy", C.c_void_p),
        ("seed", C.c_uint64),
        ("state_kind", C.c_int),
    ]


class InstanceDesc(C.Structure):
    _fields_ = [("K", C.c_int), ("T", C.c_int), ("N_r", C.c_int), ("n_track", C.c_int),
                ("half_width", C.c_float), ("track_offset", C.c_int), ("V_offset", C.c_int)]


_vp, _i, _u32, _f, _dp = C.c_void_p, C.c_int, C.c_uint32, C.c_float, C.c_void_p

_SIGS = {
    "smppi_default_params": ([C.POINTER(Params)], None),
    "smppi_create": ([C.POINTER(Params), _vp, C.POINTER(_vp)], _i),
    "smppi_destroy": ([_vp], _i),
    "smppi_last_error": ([_vp], C.c_char_p),
    "smppi_sync_status": ([_vp, C.POINTER(_u32)], _i),
    "smppi_step": ([_vp, _vp, _vp, _u32, _u32, _vp, _vp], _i),
    "smppi_update": ([_vp, _vp, _vp, _u32, _u32], _i),
    "smppi_step_partial": ([_vp, _vp, _vp, _u32, _u32, _i, _i, _vp], _i),
    "smppi_merge_partials": ([_vp, _i, _vp, _vp], _i),
    "smppi_cost_grad": ([_vp, _i, _vp, _vp, _i, _f, _f, _i, _vp, _vp], _i),
    "smppi_repair": ([_vp, _i, _vp, _vp, _vp, _i, _i, _f, _vp, _vp], _i),
    "smppi_apply": ([_vp, _vp, _vp, _vp, _u32, _u32], _i),
    "smppi_shield_update": ([_vp, _vp, _vp, _vp, _u32, _u32, _i, _vp, _i], _i),
    "smppi_shield_loop": ([_vp, _vp, _vp, _vp, _u32, _u32, _i, _i], _i),
    "smppi_debug_noise": ([_vp, _u32, _u32, _i, _i, _vp, _vp], _i),
    "smppi_debug_wait_timeout": ([_i, _vp, _vp], _i),
    "smppi_debug_elementary": ([_i, _i, _vp, _vp, _vp, _vp, _vp], _i),
    "smppi_step_noalloc": ([C.POINTER(Params), _vp, _vp, _u32, _u32, _vp, _vp], _i),
    "smppi_batch_create": ([C.POINTER(Params), _i, C.POINTER(InstanceDesc), _vp, _i, _vp,
                            C.POINTER(_vp)], _i),
    "smppi_batch_destroy": ([_vp], _i),
    "smppi_batch_last_error": ([_vp], C.c_char_p),
    "smppi_batch_step": ([_vp, _vp, _vp, _vp, _u32, _i], _i),
    "smppi_batch_loop": ([_vp, _vp, _vp, _vp, _u32, _i, _i], _i),
    "smppi_batch_sync_status": ([_vp, C.POINTER(_u32)], _i),
    "smppi_batch_config": ([_vp, C.POINTER(_i), C.POINTER(_i)], _i),
    "smppi_batch_monitor": ([_vp, _vp, _vp, _i], _i),
    "smppi_timing": ([_vp, _i], _i),
    "smppi_timing_read": ([_vp, C.POINTER(C.c_double), C.POINTER(C.c_int), _i], _i),
}

KERNEL_KINDS = ("rollout", "update", "seg0", "repair", "apply", "cost_grad", "update_shield",
                "merge")

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libsmppi.so and declare its signatures.  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("libsmppi.so not found at %s: run __graft_entry__.build() "
                              "(there is no CPU fallback)" % path)
        L = C.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return int(t)


def _check(status, handle=None):
    if status != OK:
        msg = load_library().smppi_last_error(handle)
        raise SmppiError(status, msg.decode() if msg else "")


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def default_params() -> Params:
    p = Params()
    load_library().smppi_default_params(C.byref(p))
    return p


def params_from_dict(d: dict, track_dev: torch.Tensor, max_seq: int = 1,
                     checkpoint: int = 0) -> Params:
    """smppi_params from a parameter dict (names as in inputs.DEFAULT_PARAMS)."""
    p = default_params()
    for name in ("m", "Iz", "lf", "lr", "B", "Ct", "g", "fx_gain", "dt", "gamma", "alpha",
                 "C_cbf", "q_v", "v_target", "q_d", "C_obs", "half_width", "ls_s0", "ls_c"):
        setattr(p, name, float(d[name]))
    p.lam = float(d["lam"])
    for name in ("sigma", "u_min", "u_max", "dist_sigma"):
        arr = getattr(p, name)
        arr[0], arr[1] = float(d[name][0]), float(d[name][1])
    p.K, p.T, p.N_r = int(d["K"]), int(d["T"]), int(d["N_r"])
    p.ls_max_halvings = int(d["ls_max_halvings"])
    p.checkpoint = int(checkpoint)
    p.max_seq = int(max_seq)
    p.n_track = int(track_dev.shape[0])
    p.track_xy = _ptr(track_dev)
    p.seed = int(d["seed"])
    p.state_kind = int(d.get("state_kind", 0))
    return p


# --- entry points (same names as the C ABI) ---------------------------------

def smppi_create(params: Params, stream=None) -> int:
    h = C.c_void_p()
    _check(load_library().smppi_create(C.byref(params), _stream(stream), C.byref(h)))
    return h.value


def smppi_destroy(h):
    _check(load_library().smppi_destroy(h))


def smppi_last_error(h) -> str:
    m = load_library().smppi_last_error(h)
    return m.decode() if m else ""


def smppi_sync_status(h) -> tuple[int, int]:
    bits = C.c_uint32()
    st = load_library().smppi_sync_status(h, C.byref(bits))
    return st, bits.value


def smppi_step(h, x0, V, iter=0, instance=0, S_out=None, traj_out=None):
    _check(load_library().smppi_step(h, _ptr(x0), _ptr(V), iter, instance, _ptr(S_out),
                                     _ptr(traj_out)), h)


def smppi_update(h, S, V, iter=0, instance=0):
    _check(load_library().smppi_update(h, _ptr(S), _ptr(V), iter, instance), h)


def smppi_step_partial(h, x0, V, iter, instance, k_lo, k_hi, partial_out):
    """Rollouts k_lo .. k_hi - 1 -> partial_out (float64, 2T + 2): (m, eta, A)."""
    _check(load_library().smppi_step_partial(h, _ptr(x0), _ptr(V), iter, instance, int(k_lo),
                                             int(k_hi), _ptr(partial_out)), h)


def smppi_merge_partials(h, n_parts, partials, V):
    """V <- V+ from n_parts slice partials (float64, n_parts x (2T + 2))."""
    _check(load_library().smppi_merge_partials(h, int(n_parts), _ptr(partials), _ptr(V)), h)


def shard_range(K: int, world: int, rank: int) -> tuple[int, int]:
    """The contiguous slice [k_lo, k_hi) of K rollouts that rank `rank` of
    `world` runs: sizes differ by at most one, lower ranks take the larger."""
    if world < 1 or not 0 <= rank < world or K < world:
        raise ValueError("need 1 <= world <= K and 0 <= rank < world")
    q, r = divmod(K, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def smppi_cost_grad(h, n_seq, x0, V, N, w_run, w_cbf, checkpoint, J_out, grad_out):
    _check(load_library().smppi_cost_grad(h, n_seq, _ptr(x0), _ptr(V), N, w_run, w_cbf,
                                          checkpoint, _ptr(J_out), _ptr(grad_out)), h)


def smppi_repair(h, n_seq, x0, V_in, V_out, n_iters, mode=1, delta=0.0, merit_out=None,
                 iters_out=None):
    _check(load_library().smppi_repair(h, n_seq, _ptr(x0), _ptr(V_in), _ptr(V_out), n_iters,
                                       mode, delta, _ptr(merit_out), _ptr(iters_out)), h)


def smppi_apply(h, x0, V, V_exec, n, instance=0):
    _check(load_library().smppi_apply(h, _ptr(x0), _ptr(V), _ptr(V_exec), n, instance), h)


def smppi_shield_update(h, x0, V, V_safe, iter, instance=0, n_repair=10, merit_out=None,
                        host_buffers=False):
    _check(load_library().smppi_shield_update(h, _ptr(x0), _ptr(V), _ptr(V_safe), iter, instance,
                                              n_repair, _ptr(merit_out), int(bool(host_buffers))),
           h)


def smppi_shield_loop(h, x0, V, V_safe, iter0, instance=0, n_repair=10, n_updates=1):
    _check(load_library().smppi_shield_loop(h, _ptr(x0), _ptr(V), _ptr(V_safe), iter0, instance,
                                            n_repair, n_updates), h)


def smppi_debug_noise(h, iter, instance, K, T, eps_out=None, raw_out=None):
    _check(load_library().smppi_debug_noise(h, iter, instance, K, T, _ptr(eps_out),
                                            _ptr(raw_out)), h)


def smppi_debug_wait_timeout(which, status, stream=None):
    """Self-test of the bounded device waits: a block waits on something nothing
    completes (0: an mbarrier phase, 1: a shared-memory counter), gives up and
    ORs DEV_TIMEOUT into the device word `status`."""
    _check(load_library().smppi_debug_wait_timeout(int(which), _ptr(status), _stream(stream)))


def smppi_debug_elementary(fn, a, b, out, ref, stream=None):
    """The library's elementary function `fn` (smppi.h) of a (and b) into out,
    CUDA's own into ref; device float32 tensors of equal length."""
    _check(load_library().smppi_debug_elementary(int(fn), int(a.numel()), _ptr(a), _ptr(b),
                                                 _ptr(out), _ptr(ref), _stream(stream)))


def smppi_step_noalloc(params: Params, x0, V, iter=0, instance=0, S_out=None, stream=None):
    """smppi_step without a handle and without allocating (fixed in-library scratch)."""
    _check(load_library().smppi_step_noalloc(C.byref(params), _ptr(x0), _ptr(V), iter, instance,
                                             _ptr(S_out), _stream(stream)))


def _bcheck(status, b=None):
    if status != OK:
        msg = load_library().smppi_batch_last_error(b)
        raise SmppiError(status, msg.decode() if msg else "")


def smppi_batch_create(shared: Params, descs, tracks_xy, block_rollouts=0, stream=None) -> int:
    n = len(descs)
    arr = (InstanceDesc * n)(*descs)
    b = C.c_void_p()
    _bcheck(load_library().smppi_batch_create(C.byref(shared), n, arr, _ptr(tracks_xy),
                                              int(block_rollouts), _stream(stream), C.byref(b)))
    return b.value


def smppi_batch_destroy(b):
    _bcheck(load_library().smppi_batch_destroy(b))


def smppi_batch_step(b, x0, V, V_safe, iter, n_repair=10):
    _bcheck(load_library().smppi_batch_step(b, _ptr(x0), _ptr(V), _ptr(V_safe), iter, n_repair), b)


def smppi_batch_loop(b, x0, V, V_safe, iter0, n_repair=10, n_updates=1):
    _bcheck(load_library().smppi_batch_loop(b, _ptr(x0), _ptr(V), _ptr(V_safe), iter0, n_repair,
                                            n_updates), b)


def smppi_batch_sync_status(b) -> tuple[int, int]:
    bits = C.c_uint32()
    st = load_library().smppi_batch_sync_status(b, C.byref(bits))
    return st, bits.value


def smppi_batch_config(b) -> tuple[int, int]:
    rb, grid = C.c_int(), C.c_int()
    _bcheck(load_library().smppi_batch_config(b, C.byref(rb), C.byref(grid)), b)
    return rb.value, grid.value


def smppi_batch_monitor(b, B: int, reset: bool = False):
    """(violations, outside) per problem: executed closed-loop steps that broke the
    discrete CBF condition, and that ended outside the track (uint32 arrays)."""
    viol = np.zeros(B, np.uint32)
    out = np.zeros(B, np.uint32)
    _bcheck(load_library().smppi_batch_monitor(b, viol.ctypes.data, out.ctypes.data,
                                               int(bool(reset))), b)
    return viol, out


class Batch:
    """Owns a batch handle for an inputs.InstanceBatch (device copies of tracks,
    x0, V, V_safe laid out back to back)."""

    def __init__(self, ib, block_rollouts=0, device="cuda", stream=None):
        self.device = torch.device(device)
        B = len(ib.params)
        self.B = B
        self.T = [int(t) for t in ib.T]
        self.V_off = np.concatenate([[0], np.cumsum(self.T)[:-1]]).astype(int)
        n_tr = ib.tracks.shape[1]
        self.tracks = torch.as_tensor(np.ascontiguousarray(ib.tracks.reshape(-1, 2), np.float32),
                                      device=self.device)
        descs = [InstanceDesc(int(ib.K[i]), self.T[i], self.T[i], n_tr, float(ib.w[i]),
                              i * n_tr, int(self.V_off[i])) for i in range(B)]
        self.shared = params_from_dict(ib.params[0], self.tracks)
        self.b = smppi_batch_create(self.shared, descs, self.tracks, block_rollouts, stream)
        self.x0 = torch.as_tensor(np.ascontiguousarray(ib.x0, np.float32), device=self.device)
        self.V = torch.zeros((sum(self.T), 2), dtype=torch.float32, device=self.device)
        self.V_safe = torch.zeros_like(self.V)

    def split(self, t):
        a = t.detach().cpu().numpy()
        return [a[o:o + T] for o, T in zip(self.V_off, self.T)]

    def close(self):
        if self.b:
            smppi_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def smppi_timing(h, enable: bool):
    _check(load_library().smppi_timing(h, int(bool(enable))), h)


def smppi_timing_read(h) -> dict:
    """{kind: (total ms, launches)} of the kernels timed since the last read."""
    n = len(KERNEL_KINDS)
    ms = (C.c_double * n)()
    cnt = (C.c_int * n)()
    _check(load_library().smppi_timing_read(h, ms, cnt, n), h)
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}


# --- convenience owner of one handle ---------------------------------------

class Controller:
    """Owns a handle, its device track and parameters for one problem."""

    def __init__(self, params: dict, track: np.ndarray, max_seq: int = 1, checkpoint: int = 0,
                 device="cuda", stream=None):
        self.device = torch.device(device)
        self.params = dict(params)
        self.track = torch.as_tensor(np.ascontiguousarray(track, np.float32), device=self.device)
        self.p = params_from_dict(self.params, self.track, max_seq=max_seq, checkpoint=checkpoint)
        self.K, self.T, self.max_seq = self.p.K, self.p.T, max_seq
        self.stream = stream
        self.h = smppi_create(self.p, stream)

    def close(self):
        if self.h:
            smppi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tensor(self, a, dtype=torch.float32):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=self.device).contiguous()

    def step(self, x0, V, iter=0, instance=0, want_S=False, want_traj=False):
        """V (T, 2) is updated in place to V+; returns (S or None, traj or None)."""
        S = torch.empty(self.K, device=self.device) if want_S else None
        tr = torch.empty((self.K, self.T + 1, 6), device=self.device) if want_traj else None
        smppi_step(self.h, x0, V, iter, instance, S, tr)
        return S, tr

    def sync_status(self):
        return smppi_sync_status(self.h)


class ShieldCost(torch.autograd.Function):
    """J(V) = w_run sum q + w_cbf sum C max(0, (1-alpha) h_t - h_{t+1}) per sequence,
    differentiated by the library's checkpointed reverse-mode adjoint."""

    @staticmethod
    def forward(ctx, V, x0, ctl: Controller, w_run: float = 0.0, w_cbf: float = 1.0,
                N: int | None = None, checkpoint: int = 0):
        V = V.detach().contiguous()
        n_seq = V.shape[0] if V.dim() == 3 else 1
        N = ctl.T if N is None else N
        J = torch.empty(n_seq, dtype=torch.float64, device=V.device)
        g = torch.empty_like(V)
        smppi_cost_grad(ctl.h, n_seq, x0.contiguous(), V, N, w_run, w_cbf, checkpoint, J, g)
        ctx.save_for_backward(g)
        return J.to(V.dtype)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        shape = [-1] + [1] * (g.dim() - 1) if g.dim() == 3 else [1, 1]
        return g * gJ.reshape(shape).to(g.dtype), None, None, None, None, None, None
