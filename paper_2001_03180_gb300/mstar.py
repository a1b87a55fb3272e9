"""Thin Python binding of libmstar (include/mstar.h): argument marshalling only.

Every function keeps the C name. Arrays may be numpy arrays (host) or CUDA torch
tensors (device); device memory and streams come from PyTorch. There is no CPU
fallback: if libmstar.so is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmstar.so")

MSTAR_OK = 0
MSTAR_ERR_INVALID_ARG = -1
MSTAR_ERR_NONFINITE = -2
MSTAR_ERR_NO_CONVERGENCE = -3
MSTAR_ERR_TIMEOUT = -4
MSTAR_ERR_CUDA = -5
MSTAR_ERR_UNSUPPORTED = -6
MSTAR_ERR_NOMEM = -7
MSTAR_MAX_N = 10240

# Names the header declares (checked by the tests against the library's exports).
EXPORTS = [
    "mstar_default_params", "mstar_workspace_bytes", "mstar_init", "mstar_step", "mstar_attempt",
    "mstar_energy", "mstar_get_state", "mstar_set_state", "mstar_set_H", "mstar_get_mst",
    "mstar_accelerations", "mstar_tune_pair_tile", "mstar_free", "mstar_strerror", "mstar_launch_count",
    "mstar_profile_enable", "mstar_profile_read", "mstar_fp64_fma_rate", "mstar_accelerations_noalloc",
    "mstar_batch_workspace_bytes", "mstar_batch_init", "mstar_step_batched", "mstar_batch_get_state",
    "mstar_batch_set_H", "mstar_batch_set_schedule", "mstar_batch_get_schedule", "mstar_batch_autotune",
    "mstar_batch_launch_count", "mstar_batch_free",
    "mstar_adjoint_forward", "mstar_step_adjoint", "mstar_adjoint_free", "mstar_rebuild_test",
]
MSTAR_BATCH_MAX_N = 512
MSTAR_BATCH_NUM_CLASSES = 7
MSTAR_NOALLOC_MAX_N = 2048


class mstar_params(C.Structure):
    _fields_ = [("eta_gbs", C.c_double), ("a_gbs", C.c_double), ("fac_min", C.c_double),
                ("fac_max", C.c_double), ("q_first", C.c_double), ("t_tol", C.c_double),
                ("G", C.c_double), ("k_fix", C.c_int), ("n_d", C.c_int), ("max_halvings", C.c_int),
                ("max_time_iter", C.c_int), ("mst_method", C.c_int), ("mst_nsub", C.c_int),
                ("pair_tile", C.c_int), ("pair_split", C.c_int), ("division_schedule", C.c_int), ("division_cluster", C.c_int)]


class mstar_stats(C.Structure):
    _fields_ = [("accepted", C.c_longlong), ("rejected", C.c_longlong), ("force_evals", C.c_longlong),
                ("time_iters", C.c_longlong), ("eps_last", C.c_double), ("H", C.c_double),
                ("t", C.c_double)]


class mstar_batch_stats(C.Structure):
    _fields_ = [("accepted", C.c_longlong), ("rejected", C.c_longlong), ("force_evals", C.c_longlong),
                ("finished", C.c_int), ("failed", C.c_int)]


class mstar_profile(C.Structure):
    _fields_ = [("pair_launches", C.c_longlong), ("pair_ms", C.c_double),
                ("pair_interactions", C.c_double), ("force_evals", C.c_longlong)]


_lib = None


class MstarError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {mstar_strerror(code)} ({code})")
        self.code = code


def load():
    """Load libmstar.so (no fallback of any kind)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmstar.so not built ({LIB_PATH}); run paper_2001_03180_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.c_void_p, C.c_void_p
    L.mstar_default_params.argtypes = [C.POINTER(mstar_params)]
    L.mstar_default_params.restype = None
    L.mstar_workspace_bytes.argtypes = [C.c_int, C.POINTER(mstar_params)]
    L.mstar_workspace_bytes.restype = C.c_size_t
    L.mstar_init.argtypes = [C.POINTER(vp), C.c_int, dp, dp, dp, C.POINTER(mstar_params), vp, C.c_size_t, vp]
    L.mstar_step.argtypes = [vp, C.c_double, C.c_int, C.POINTER(mstar_stats)]
    L.mstar_attempt.argtypes = [vp, C.c_double, C.POINTER(C.c_double), dp, dp, C.POINTER(C.c_double)]
    L.mstar_energy.argtypes = [vp] + [C.POINTER(C.c_double)] * 3 + [dp, dp]
    L.mstar_get_state.argtypes = [vp, C.POINTER(C.c_double), dp, dp]
    L.mstar_set_state.argtypes = [vp, C.c_double, dp, dp]
    L.mstar_set_H.argtypes = [vp, C.c_double]
    L.mstar_get_mst.argtypes = [vp, ip, ip, ip, ip]
    L.mstar_accelerations.argtypes = [vp, dp, C.POINTER(C.c_double)]
    L.mstar_tune_pair_tile.argtypes = [C.c_int, dp, dp, dp, C.POINTER(mstar_params), C.c_int, C.POINTER(C.c_int),
                                       C.POINTER(C.c_int), dp, vp]
    L.mstar_free.argtypes = [vp]
    L.mstar_free.restype = None
    L.mstar_strerror.argtypes = [C.c_int]
    L.mstar_strerror.restype = C.c_char_p
    L.mstar_launch_count.argtypes = [vp]
    L.mstar_launch_count.restype = C.c_longlong
    L.mstar_profile_enable.argtypes = [vp, C.c_int]
    L.mstar_profile_read.argtypes = [vp, C.POINTER(mstar_profile)]
    L.mstar_fp64_fma_rate.argtypes = [C.POINTER(C.c_double), vp]
    L.mstar_accelerations_noalloc.argtypes = [C.c_int, dp, dp, C.c_double, dp, dp, vp]
    L.mstar_batch_workspace_bytes.argtypes = [C.c_int, ip, C.POINTER(mstar_params)]
    L.mstar_batch_workspace_bytes.restype = C.c_size_t
    L.mstar_batch_init.argtypes = [C.POINTER(vp), C.c_int, ip, dp, dp, dp, C.POINTER(mstar_params), vp, C.c_size_t, vp]
    L.mstar_step_batched.argtypes = [vp, C.c_double, C.c_int, C.POINTER(mstar_batch_stats)]
    L.mstar_batch_get_state.argtypes = [vp, dp, dp, dp, dp, ip]
    L.mstar_batch_set_H.argtypes = [vp, dp]
    L.mstar_batch_set_schedule.argtypes = [vp, ip]
    L.mstar_batch_get_schedule.argtypes = [vp, ip]
    L.mstar_batch_autotune.argtypes = [vp, C.c_double, C.c_int, ip, C.POINTER(C.c_double)]
    L.mstar_batch_launch_count.argtypes = [vp]
    L.mstar_batch_launch_count.restype = C.c_longlong
    L.mstar_batch_free.argtypes = [vp]
    L.mstar_batch_free.restype = None
    L.mstar_adjoint_forward.argtypes = [vp, C.c_double, C.c_int, C.c_int, C.POINTER(vp)]
    L.mstar_step_adjoint.argtypes = [vp, vp, dp, dp, C.c_double, dp, dp, dp]
    L.mstar_adjoint_free.argtypes = [vp]
    L.mstar_adjoint_free.restype = None
    L.mstar_rebuild_test.argtypes = [C.c_int, C.c_int, dp, dp, dp, ip, ip, C.c_int, C.c_int, C.c_int, ip, dp, dp, dp,
                                     ip, dp, vp]
    _lib = L
    return L


def _ptr(x):
    """Data pointer of a numpy array or a torch tensor (host or device); None -> NULL."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if isinstance(x, C.c_void_p):
        return x.value
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _check(rc, where):
    if rc != MSTAR_OK:
        raise MstarError(rc, where)


def mstar_strerror(code: int) -> str:
    return load().mstar_strerror(int(code)).decode()


def _system(m, r, v):
    """Contiguous float64 m[n], r[n, 3], v[n, 3] of one system. The library reads exactly n
    masses and 3n coordinates through each pointer, so any other shape is a ValueError
    (r and v may also come flat, as 3n values in body order)."""
    m = np.ascontiguousarray(m, dtype=np.float64)
    if m.ndim != 1:
        raise ValueError(f"masses must be a vector, got shape {m.shape}")
    return m, _vectors(r, len(m), "r"), _vectors(v, len(m), "v")


def _vectors(x, n, name):
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.shape not in ((n, 3), (3 * n,)):
        raise ValueError(f"{name} must have shape ({n}, 3), got {x.shape}")
    return x.reshape(n, 3)


def mstar_default_params(**overrides) -> mstar_params:
    p = mstar_params()
    load().mstar_default_params(C.byref(p))
    names = {f[0] for f in mstar_params._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise TypeError(f"unknown mstar_params field {k!r}")
        setattr(p, k, v)
    return p


def mstar_workspace_bytes(n: int, p: mstar_params | None = None) -> int:
    return load().mstar_workspace_bytes(int(n), C.byref(p) if p is not None else None)


def mstar_init(n, m, r, v, p=None, workspace=None, workspace_bytes=0, cuda_stream=None):
    ctx = C.c_void_p()
    rc = load().mstar_init(C.byref(ctx), int(n), _ptr(m), _ptr(r), _ptr(v), C.byref(p) if p is not None else None,
                           _ptr(workspace), int(workspace_bytes), cuda_stream)
    _check(rc, "mstar_init")
    return ctx


def mstar_step(ctx, t_end, max_gbs_steps):
    st = mstar_stats()
    rc = load().mstar_step(ctx, float(t_end), int(max_gbs_steps), C.byref(st))
    return rc, st


def mstar_attempt(ctx, H, r_out=None, v_out=None):
    eps = C.c_double()
    t = C.c_double()
    rc = load().mstar_attempt(ctx, float(H), C.byref(eps), _ptr(r_out), _ptr(v_out), C.byref(t))
    _check(rc, "mstar_attempt")
    return eps.value, t.value


def mstar_energy(ctx, P=None, L=None):
    E, T, U = C.c_double(), C.c_double(), C.c_double()
    rc = load().mstar_energy(ctx, C.byref(E), C.byref(T), C.byref(U), _ptr(P), _ptr(L))
    _check(rc, "mstar_energy")
    return E.value, T.value, U.value


def mstar_get_state(ctx, r=None, v=None):
    t = C.c_double()
    _check(load().mstar_get_state(ctx, C.byref(t), _ptr(r), _ptr(v)), "mstar_get_state")
    return t.value


def mstar_set_state(ctx, t, r, v):
    _check(load().mstar_set_state(ctx, float(t), _ptr(r), _ptr(v)), "mstar_set_state")


def mstar_set_H(ctx, H):
    _check(load().mstar_set_H(ctx, float(H)), "mstar_set_H")


def mstar_get_mst(ctx, root=None, parent=None, level=None, order=None):
    _check(load().mstar_get_mst(ctx, _ptr(root), _ptr(parent), _ptr(level), _ptr(order)), "mstar_get_mst")


def mstar_accelerations(ctx, a=None):
    U = C.c_double()
    _check(load().mstar_accelerations(ctx, _ptr(a), C.byref(U)), "mstar_accelerations")
    return U.value


def mstar_tune_pair_tile(m, r, v, repeats=3, cuda_stream=None, **params):
    """The pair loop whose GBS step attempts run fastest on the system (m, r, v) under the given
    parameters: returns ((tile, split), {(tile, split): ms per attempt}) over (32, 4), (32, 1),
    (64, 1) and (128, 1)."""
    m, r, v = _system(m, r, v)
    p = mstar_default_params(**params)
    tile, split = C.c_int(), C.c_int()
    ms = np.zeros(4)
    rc = load().mstar_tune_pair_tile(len(m), _ptr(m), _ptr(r), _ptr(v), C.byref(p), int(repeats), C.byref(tile),
                                     C.byref(split), _ptr(ms), cuda_stream)
    _check(rc, "mstar_tune_pair_tile")
    keys = [(32, 4), (32, 1), (64, 1), (128, 1)]
    return (tile.value, split.value), {k: float(x) for k, x in zip(keys, ms)}


def mstar_free(ctx):
    if ctx:
        load().mstar_free(ctx)


def mstar_launch_count(ctx) -> int:
    return load().mstar_launch_count(ctx)


def mstar_profile_enable(ctx, on: bool):
    _check(load().mstar_profile_enable(ctx, int(bool(on))), "mstar_profile_enable")


def mstar_profile_read(ctx) -> mstar_profile:
    pr = mstar_profile()
    _check(load().mstar_profile_read(ctx, C.byref(pr)), "mstar_profile_read")
    return pr


def mstar_fp64_fma_rate(cuda_stream=None) -> float:
    r = C.c_double()
    _check(load().mstar_fp64_fma_rate(C.byref(r), cuda_stream), "mstar_fp64_fma_rate")
    return r.value


def mstar_accelerations_noalloc(n, m, r, G, a, U, cuda_stream=None) -> int:
    """Allocation-free pair loop; m, r, a, U are device tensors. Returns the status code."""
    return load().mstar_accelerations_noalloc(int(n), _ptr(m), _ptr(r), float(G), _ptr(a), _ptr(U),
                                              cuda_stream)


class Integrator:
    """One N-body system on the GPU. Device memory (the context workspace) is a torch
    tensor; all GPU work runs on the torch stream current at construction."""

    def __init__(self, m, r, v, device=None, **params):
        import torch

        m, r, v = _system(m, r, v)
        if not torch.cuda.is_available():
            raise RuntimeError("libmstar needs a CUDA GPU")
        load()
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.p = mstar_default_params(**params)
        self.n = len(m)
        nbytes = mstar_workspace_bytes(self.n, self.p)
        if nbytes == 0:
            raise MstarError(MSTAR_ERR_INVALID_ARG, "mstar_workspace_bytes")
        with torch.cuda.device(self.device):
            self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            off = (-self.ws.data_ptr()) % 256
            self._ws_ptr = self.ws.data_ptr() + off
            self.stream = torch.cuda.current_stream(self.device)
            self.ctx = C.c_void_p()
            rc = load().mstar_init(C.byref(self.ctx), self.n, _ptr(m), _ptr(r), _ptr(v), C.byref(self.p),
                                   C.c_void_p(self._ws_ptr), nbytes, C.c_void_p(self.stream.cuda_stream))
            _check(rc, "mstar_init")

    def close(self):
        if getattr(self, "ctx", None):
            mstar_free(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()

    def step(self, t_end, max_steps=1 << 30, check=True):
        rc, st = mstar_step(self.ctx, t_end, max_steps)
        if check:
            _check(rc, "mstar_step")
        return rc, dict(accepted=st.accepted, rejected=st.rejected, force_evals=st.force_evals,
                        time_iters=st.time_iters, eps_last=st.eps_last, H=st.H, t=st.t)

    def attempt(self, H):
        r = np.empty((self.n, 3))
        v = np.empty((self.n, 3))
        eps, t = mstar_attempt(self.ctx, H, r, v)
        return dict(eps=eps, r=r, v=v, t=t)

    def state(self):
        r = np.empty((self.n, 3))
        v = np.empty((self.n, 3))
        t = mstar_get_state(self.ctx, r, v)
        return dict(t=t, r=r, v=v)

    def set_state(self, t, r, v):
        mstar_set_state(self.ctx, t, _vectors(r, self.n, "r"), _vectors(v, self.n, "v"))

    def set_H(self, H):
        mstar_set_H(self.ctx, H)

    def mst(self, with_order=True):
        """(root, parent, level, order); with_order=False returns the step builder's tree
        and order None."""
        root = np.zeros(1, np.int32)
        parent = np.empty(self.n, np.int32)
        level = np.empty(self.n, np.int32)
        order = np.empty(self.n, np.int32) if with_order else None
        mstar_get_mst(self.ctx, root, parent, level, order)
        return int(root[0]), parent, level, order

    def accelerations(self):
        a = np.empty((self.n, 3))
        U = mstar_accelerations(self.ctx, a)
        return a, U

    def energy(self):
        P = np.empty(3)
        L = np.empty(3)
        E, T, U = mstar_energy(self.ctx, P, L)
        return dict(E=E, T=T, U=U, P=P, L=L)


def mstar_batch_workspace_bytes(nsys, offsets, p=None) -> int:
    offsets = np.ascontiguousarray(offsets, dtype=np.int32)
    return load().mstar_batch_workspace_bytes(int(nsys), _ptr(offsets), C.byref(p) if p is not None else None)


def mstar_batch_init(nsys, offsets, m, r, v, p=None, workspace=None, workspace_bytes=0, cuda_stream=None):
    offsets = np.ascontiguousarray(offsets, dtype=np.int32)
    b = C.c_void_p()
    rc = load().mstar_batch_init(C.byref(b), int(nsys), _ptr(offsets), _ptr(m), _ptr(r), _ptr(v),
                                 C.byref(p) if p is not None else None, _ptr(workspace), int(workspace_bytes),
                                 cuda_stream)
    _check(rc, "mstar_batch_init")
    return b


def mstar_step_batched(b, t_end, launches):
    st = mstar_batch_stats()
    rc = load().mstar_step_batched(b, float(t_end), int(launches), C.byref(st))
    return rc, st


def mstar_batch_get_state(b, t=None, r=None, v=None, eps=None, status=None):
    _check(load().mstar_batch_get_state(b, _ptr(t), _ptr(r), _ptr(v), _ptr(eps), _ptr(status)),
           "mstar_batch_get_state")


def mstar_batch_set_H(b, H):
    H = np.ascontiguousarray(H, dtype=np.float64)
    _check(load().mstar_batch_set_H(b, _ptr(H)), "mstar_batch_set_H")


def mstar_batch_set_schedule(b, schedule):
    sc = np.ascontiguousarray(schedule, dtype=np.int32)
    if sc.shape != (MSTAR_BATCH_NUM_CLASSES,):
        raise ValueError(f"schedule needs {MSTAR_BATCH_NUM_CLASSES} entries")
    _check(load().mstar_batch_set_schedule(b, _ptr(sc)), "mstar_batch_set_schedule")


def mstar_batch_get_schedule(b):
    sc = np.zeros(MSTAR_BATCH_NUM_CLASSES, np.int32)
    _check(load().mstar_batch_get_schedule(b, _ptr(sc)), "mstar_batch_get_schedule")
    return sc


def mstar_batch_autotune(b, t_end, repeats=2):
    sc = np.zeros(MSTAR_BATCH_NUM_CLASSES, np.int32)
    ms = C.c_double()
    _check(load().mstar_batch_autotune(b, float(t_end), int(repeats), _ptr(sc), C.byref(ms)), "mstar_batch_autotune")
    return sc, ms.value


def mstar_batch_launch_count(b) -> int:
    return load().mstar_batch_launch_count(b)


def mstar_batch_free(b):
    if b:
        load().mstar_batch_free(b)


class Batch:
    """Many independent systems integrated together (one or four CTAs per system per launch); device
    memory from torch, work on the torch stream current at construction."""

    def __init__(self, systems, device=None, **params):
        import torch

        systems = [_system(*sm) for sm in systems]
        if not systems:
            raise MstarError(MSTAR_ERR_INVALID_ARG, "Batch: no systems")
        if not torch.cuda.is_available():
            raise RuntimeError("libmstar needs a CUDA GPU")
        load()
        self.device = torch.device(device or "cuda")
        self.p = mstar_default_params(**params)
        sizes = [len(sm[0]) for sm in systems]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
        self.nsys = len(systems)
        self.nbody = int(self.offsets[-1])
        m = np.ascontiguousarray(np.concatenate([s[0] for s in systems]))
        r = np.ascontiguousarray(np.concatenate([s[1] for s in systems]))
        v = np.ascontiguousarray(np.concatenate([s[2] for s in systems]))
        nbytes = mstar_batch_workspace_bytes(self.nsys, self.offsets, self.p)
        if nbytes == 0:  # let the library name the problem (it rejects before allocating)
            self.b = mstar_batch_init(self.nsys, self.offsets, m, r, v, self.p)
            raise MstarError(MSTAR_ERR_INVALID_ARG, "mstar_batch_workspace_bytes")
        with torch.cuda.device(self.device):
            self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            ptr = self.ws.data_ptr() + (-self.ws.data_ptr()) % 256
            self.stream = torch.cuda.current_stream(self.device)
            self.b = mstar_batch_init(self.nsys, self.offsets, m, r, v, self.p, C.c_void_p(ptr), nbytes,
                                      C.c_void_p(self.stream.cuda_stream))

    def close(self):
        if getattr(self, "b", None):
            mstar_batch_free(self.b)
            self.b = None

    def __del__(self):
        self.close()

    def step(self, t_end, launches=1):
        rc, st = mstar_step_batched(self.b, t_end, launches)
        _check(rc, "mstar_step_batched")
        return dict(accepted=st.accepted, rejected=st.rejected, force_evals=st.force_evals,
                    finished=st.finished, failed=st.failed)

    def state(self):
        t = np.empty(self.nsys)
        eps = np.empty(self.nsys)
        status = np.empty(self.nsys, np.int32)
        r = np.empty((self.nbody, 3))
        v = np.empty((self.nbody, 3))
        mstar_batch_get_state(self.b, t, r, v, eps, status)
        o = self.offsets
        return dict(t=t, eps=eps, status=status, r=[r[o[s]:o[s + 1]] for s in range(self.nsys)],
                    v=[v[o[s]:o[s + 1]] for s in range(self.nsys)])

    def set_H(self, H):
        H = np.ascontiguousarray(H, dtype=np.float64)
        if H.shape != (self.nsys,):
            raise ValueError(f"H must have one entry per system ({self.nsys}), got shape {H.shape}")
        mstar_batch_set_H(self.b, H)

    def set_schedule(self, schedule):
        mstar_batch_set_schedule(self.b, schedule)

    def schedule(self):
        return mstar_batch_get_schedule(self.b)

    def autotune(self, t_end, repeats=2):
        """(schedule, ms of one launch) chosen by the library's autotuner; state unchanged."""
        return mstar_batch_autotune(self.b, t_end, repeats)


# ---------------------------------------------------------------- adjoint of a fixed-step run

def mstar_adjoint_forward(ctx, H, nsteps, checkpoint_every):
    a = C.c_void_p()
    _check(load().mstar_adjoint_forward(ctx, float(H), int(nsteps), int(checkpoint_every), C.byref(a)),
           "mstar_adjoint_forward")
    return a


def mstar_step_adjoint(ctx, a, g_r=None, g_v=None, g_E=0.0, d_r=None, d_v=None, d_m=None):
    _check(load().mstar_step_adjoint(ctx, a, _ptr(g_r), _ptr(g_v), float(g_E), _ptr(d_r), _ptr(d_v), _ptr(d_m)),
           "mstar_step_adjoint")


def mstar_adjoint_free(a):
    if a:
        load().mstar_adjoint_free(a)


class FixedRun:
    """nsteps GBS steps of fixed fictitious step H from (m, r, v) (numpy arrays or float64
    torch tensors, host or device), with checkpoints for the reverse sweep. `final` holds
    r, v (n x 3) and E of the final state; backward() gives the gradients of a loss with
    respect to m, r, v from its gradients with respect to the final r, v and E."""

    def __init__(self, m, r, v, H, nsteps, checkpoint_every=10, device=None, **params):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libmstar needs a CUDA GPU")
        load()
        self.torch = torch
        self.device = torch.device(device or "cuda")
        t = lambda x, shape: torch.as_tensor(x, dtype=torch.float64).reshape(shape).contiguous()  # noqa: E731
        n = int(torch.as_tensor(m).numel())
        self.n = n
        m, r, v = t(m, (n,)), t(r, (n, 3)), t(v, (n, 3))
        self.p = mstar_default_params(**params)
        nbytes = mstar_workspace_bytes(n, self.p)
        if nbytes == 0:
            raise MstarError(MSTAR_ERR_INVALID_ARG, "mstar_workspace_bytes")
        self.a = None
        self.ctx = None
        with torch.cuda.device(self.device):
            self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            ptr = self.ws.data_ptr() + (-self.ws.data_ptr()) % 256
            self.stream = torch.cuda.current_stream(self.device)
            ctx = C.c_void_p()
            _check(load().mstar_init(C.byref(ctx), n, _ptr(m), _ptr(r), _ptr(v), C.byref(self.p), C.c_void_p(ptr),
                                     nbytes, C.c_void_p(self.stream.cuda_stream)), "mstar_init")
            self.ctx = ctx
            self.a = mstar_adjoint_forward(self.ctx, H, nsteps, checkpoint_every)
            rf = torch.empty((n, 3), dtype=torch.float64, device=self.device)
            vf = torch.empty((n, 3), dtype=torch.float64, device=self.device)
            tf = mstar_get_state(self.ctx, rf, vf)
            E, T, U = mstar_energy(self.ctx, np.empty(3), np.empty(3))
        self.final = dict(r=rf, v=vf, E=E, t=tf)

    def backward(self, g_r=None, g_v=None, g_E=0.0):
        torch = self.torch
        prep = lambda g: None if g is None else torch.as_tensor(g, dtype=torch.float64, device=self.device).reshape(  # noqa: E731
            self.n, 3).contiguous()
        g_r, g_v = prep(g_r), prep(g_v)
        d_r = torch.empty((self.n, 3), dtype=torch.float64, device=self.device)
        d_v = torch.empty((self.n, 3), dtype=torch.float64, device=self.device)
        d_m = torch.empty((self.n,), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            mstar_step_adjoint(self.ctx, self.a, g_r, g_v, float(g_E), d_r, d_v, d_m)
        return d_m, d_r, d_v

    def close(self):
        if getattr(self, "a", None):
            mstar_adjoint_free(self.a)
            self.a = None
        if getattr(self, "ctx", None):
            mstar_free(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()


def fixed_run(m, r, v, H, nsteps, checkpoint_every=10, **params):
    """Differentiable fixed-step run: (r_f, v_f, E_f) = run(m, r, v) as torch tensors on the
    GPU; gradients flow to m, r, v through the library's reverse sweep."""
    import torch

    class _FixedRunFn(torch.autograd.Function):
        @staticmethod
        def forward(fctx, m_, r_, v_):
            run = FixedRun(m_.detach(), r_.detach(), v_.detach(), H, nsteps, checkpoint_every,
                           device=r_.device if r_.is_cuda else None, **params)
            fctx.run = run
            fctx.in_device = r_.device
            E = torch.tensor(run.final["E"], dtype=torch.float64, device=run.device)
            return run.final["r"].clone(), run.final["v"].clone(), E

        @staticmethod
        def backward(fctx, g_r, g_v, g_E):
            run = fctx.run
            d_m, d_r, d_v = run.backward(g_r, g_v, 0.0 if g_E is None else float(g_E))
            dev = fctx.in_device
            return d_m.to(dev), d_r.to(dev), d_v.to(dev)

    t = lambda x: torch.as_tensor(x, dtype=torch.float64)  # noqa: E731
    return _FixedRunFn.apply(t(m), t(r), t(v))


# ---------------------------------------------------------------- rebuild test (Sec. 3.5)

MSTAR_REBUILD_MAX_N = 1024


def mstar_rebuild_test(systems, coords, deconstruct, cycles, topo_every, sample_at, cuda_stream=None):
    """Jobs j = (systems[j] = (m, r, v), coords[j] (0 MST, 1 chain), deconstruct[j] (0 path sums
    and the COM shift, 1 path sums and the root kept, 2 from the root outwards, 3 from the root
    outwards and the COM shift)), all with the same n.
    Returns dict(E (jobs x samples), r, v (jobs x n x 3), topo_changes, mean_level)."""
    nj = len(systems)
    n = len(systems[0][0])
    m = np.ascontiguousarray(np.stack([np.asarray(s[0], np.float64) for s in systems]))
    r = np.ascontiguousarray(np.stack([np.asarray(s[1], np.float64).reshape(n, 3) for s in systems]))
    v = np.ascontiguousarray(np.stack([np.asarray(s[2], np.float64).reshape(n, 3) for s in systems]))
    co = np.ascontiguousarray(coords, dtype=np.int32)
    de = np.ascontiguousarray(deconstruct, dtype=np.int32)
    sa = np.ascontiguousarray(sample_at, dtype=np.int32)
    E = np.empty((nj, len(sa)))
    ro = np.empty_like(r)
    vo = np.empty_like(v)
    tc = np.empty(nj, np.int32)
    ml = np.empty(nj)
    _check(load().mstar_rebuild_test(nj, n, _ptr(m), _ptr(r), _ptr(v), _ptr(co), _ptr(de), int(cycles),
                                     int(topo_every), len(sa), _ptr(sa), _ptr(E), _ptr(ro), _ptr(vo), _ptr(tc),
                                     _ptr(ml), cuda_stream), "mstar_rebuild_test")
    return dict(E=E, r=ro, v=vo, topo_changes=tc, mean_level=ml)
