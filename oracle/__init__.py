"""Python access to the MSTAR CPU oracle (plain C, FP64). TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg import this
package. It compiles `mstar_oracle.c` with gcc on first use (or via `build()`), with
-ffp-contract=off so that the arithmetic is exactly the C source's.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mstar_oracle.c")
_LIB = os.path.join(_HERE, "libmstar_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/libmstar_oracle.so (with OpenMP if available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mstar_oracle.h"))):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
            "-o", _LIB + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("eta", C.c_double), ("a_gbs", C.c_double), ("fac_min", C.c_double),
                ("fac_max", C.c_double), ("q_first", C.c_double), ("t_tol", C.c_double),
                ("G", C.c_double), ("k_fix", C.c_int), ("n_d", C.c_int),
                ("max_halvings", C.c_int), ("max_time_iter", C.c_int), ("mst_method", C.c_int),
                ("mst_nsub", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("accepted", C.c_longlong), ("rejected", C.c_longlong),
                ("force_evals", C.c_longlong), ("time_iters", C.c_longlong),
                ("eps_last", C.c_double), ("H", C.c_double), ("t", C.c_double)]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.orc_params_default.argtypes = [C.POINTER(Params)]
            L.orc_kinetic.restype = C.c_double
            L.orc_kinetic.argtypes = [C.c_int, _D, _D]
            L.orc_potential.restype = C.c_double
            L.orc_potential.argtypes = [C.c_int, _D, _D, C.c_double]
            L.orc_com_shift.argtypes = [C.c_int, _D, _D]
            L.orc_prim.restype = C.c_int
            L.orc_prim.argtypes = [C.c_int, _D, _I, _I, _I]
            L.orc_chain.restype = C.c_int
            L.orc_chain.argtypes = [C.c_int, _D, _I, _I, _I]
            L.orc_energy_comp.restype = C.c_double
            L.orc_energy_comp.argtypes = [C.c_int, _D, _D, _D, C.c_double]
            L.orc_rebuild_run.restype = C.c_int
            L.orc_rebuild_run.argtypes = [C.c_int, _D, _D, _D, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _I, _D, _I,
                                          _D]
            L.orc_dc_mst.restype = C.c_int
            L.orc_dc_mst.argtypes = [C.c_int, _D, C.c_int, _I, _I, _I, _I, _I]
            L.orc_is_near.restype = C.c_int
            L.orc_is_near.argtypes = [_I, _I, C.c_int, C.c_int, C.c_int]
            L.orc_near_sep.argtypes = [_I, _I, _D, C.c_int, C.c_int, _D]
            L.orc_to_mst.argtypes = [C.c_int, _I, _D, _D]
            L.orc_from_mst.argtypes = [C.c_int, _D, _I, _D, _D]
            L.orc_forces.argtypes = [C.c_int, _D, C.c_double, _I, _I, C.c_int, _D, _D, _D, _D]
            L.orc_neville.argtypes = [C.c_int, _I, C.c_int, _D, _D, _D]
            L.orc_div_assign.restype = C.c_int
            L.orc_div_assign.argtypes = [C.c_int, C.c_int, _I]
            L.orc_gbs_harmonic.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int, _D, _D]
            L.orc_gbs_error.restype = C.c_double
            L.orc_gbs_error.argtypes = [C.c_int, _I, _D, _D, _D, _D, _D, C.c_double, C.c_double, C.c_double,
                                        C.c_double, C.c_double, C.c_int]
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.c_int, _D, _D, _D, C.POINTER(Params)]
            L.orc_free.argtypes = [C.c_void_p]
            L.orc_get_state.argtypes = [C.c_void_p, _D, _D, _D, _D, _D]
            L.orc_set_H.argtypes = [C.c_void_p, C.c_double]
            L.orc_attempt.restype = C.c_int
            L.orc_attempt.argtypes = [C.c_void_p, C.c_double, _D, _D, _D, _D, _D]
            L.orc_leapfrog.restype = C.c_int
            L.orc_leapfrog.argtypes = [C.c_void_p, C.c_int, C.c_double, _D, _D, _D]
            L.orc_set_state.argtypes = [C.c_void_p, C.c_double, _D, _D]
            L.orc_integrate.restype = C.c_int
            L.orc_integrate.argtypes = [C.c_void_p, C.c_double, C.c_int, C.POINTER(Stats)]
            L.orc_energy.argtypes = [C.c_void_p, _D, _D, _D, _D, _D]
            L.orc_fixed_run.restype = C.c_int
            L.orc_fixed_run.argtypes = [C.c_void_p, C.c_double, C.c_int]
            L.orc_fixed_run_tl.restype = C.c_int
            L.orc_fixed_run_tl.argtypes = [C.c_int, _D, _D, _D, _D, _D, _D, C.POINTER(Params), C.c_double,
                                           C.c_int, _D, _D, _D, _D, _D, _D]
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_get_threads.restype = C.c_int
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _i(a):
    return a.ctypes.data_as(_I)


def _f64(x, shape=None):
    a = np.ascontiguousarray(x, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def default_params(**kw) -> Params:
    p = Params()
    lib().orc_params_default(C.byref(p))
    names = {f[0] for f in Params._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown oracle parameter {k!r}")
        setattr(p, k, v)
    return p


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def kinetic(m, v) -> float:
    m = _f64(m); v = _f64(v, (-1, 3))
    return lib().orc_kinetic(len(m), _d(m), _d(v))


def potential(m, r, G=1.0) -> float:
    m = _f64(m); r = _f64(r, (-1, 3))
    return lib().orc_potential(len(m), _d(m), _d(r), G)


def com_shift(m, w):
    m = _f64(m); w = _f64(w, (-1, 3)).copy()
    lib().orc_com_shift(len(m), _d(m), _d(w))
    return w


def prim(r):
    r = _f64(r, (-1, 3))
    n = r.shape[0]
    parent = np.empty(n, np.int32); level = np.empty(n, np.int32); order = np.empty(n, np.int32)
    root = lib().orc_prim(n, _d(r), _i(parent), _i(level), _i(order))
    return root, parent, level, order


def chain(r):
    """Chained coordinates (Sec. 2.2) as a tree rooted at the tail: (tail, parent, level, order)."""
    r = _f64(r, (-1, 3))
    n = r.shape[0]
    parent = np.empty(n, np.int32); level = np.empty(n, np.int32); order = np.empty(n, np.int32)
    tail = lib().orc_chain(n, _d(r), _i(parent), _i(level), _i(order))
    return tail, parent, level, order


def energy_comp(m, r, v, G=1.0) -> float:
    m = _f64(m); n = len(m)
    return lib().orc_energy_comp(n, _d(m), _d(_f64(r, (n, 3))), _d(_f64(v, (n, 3))), float(G))


def rebuild_run(m, r, v, coords, cycles, topo_every, sample_at, deconstruct=0):
    """Rebuild test of Sec. 3.5 (coords 0: MST, 1: chain; deconstruct 0: path sums and the COM
    shift, 1: path sums and the root kept, 2: root outwards from the kept root, 3: root outwards
    and the COM shift). Returns dict(r, v, E, topo_changes, mean_level); E[s] after sample_at[s]
    cycles."""
    m = _f64(m); n = len(m)
    r = _f64(r, (n, 3)).copy(); v = _f64(v, (n, 3)).copy()
    sa = np.ascontiguousarray(sample_at, dtype=np.int32)
    E = np.empty(len(sa)); ch = np.zeros(1, np.int32); ml = np.zeros(1)
    rc = lib().orc_rebuild_run(n, _d(m), _d(r), _d(v), int(coords), int(deconstruct), int(cycles), int(topo_every),
                               len(sa), _i(sa), _d(E), _i(ch), _d(ml))
    if rc != 0:
        raise ValueError(f"orc_rebuild_run failed ({rc})")
    return dict(r=r, v=v, E=E, topo_changes=int(ch[0]), mean_level=float(ml[0]))


def dc_mst(r, leaf_cap=0):
    """Divide-and-conquer spanning tree (Sec. 3.3): (root, parent, level, order, leaf_of, nleaf)."""
    r = _f64(r, (-1, 3))
    n = r.shape[0]
    parent = np.empty(n, np.int32); level = np.empty(n, np.int32); order = np.empty(n, np.int32)
    leaf = np.empty(n, np.int32); nleaf = np.zeros(1, np.int32)
    root = lib().orc_dc_mst(n, _d(r), int(leaf_cap), _i(parent), _i(level), _i(order), _i(leaf), _i(nleaf))
    return root, parent, level, order, leaf, int(nleaf[0])


def is_near(parent, level, i, j, n_d=2) -> bool:
    parent = np.ascontiguousarray(parent, np.int32); level = np.ascontiguousarray(level, np.int32)
    return bool(lib().orc_is_near(_i(parent), _i(level), int(i), int(j), int(n_d)))


def near_sep(parent, level, X, i, j):
    parent = np.ascontiguousarray(parent, np.int32); level = np.ascontiguousarray(level, np.int32)
    X = _f64(X, (-1, 3)); d = np.empty(3)
    lib().orc_near_sep(_i(parent), _i(level), _d(X), int(i), int(j), _d(d))
    return d


def to_mst(parent, w):
    parent = np.ascontiguousarray(parent, np.int32); w = _f64(w, (-1, 3)); W = np.empty_like(w)
    lib().orc_to_mst(len(parent), _i(parent), _d(w), _d(W))
    return W


def from_mst(m, parent, W):
    m = _f64(m); parent = np.ascontiguousarray(parent, np.int32); W = _f64(W, (-1, 3)); w = np.empty_like(W)
    lib().orc_from_mst(len(m), _d(m), _i(parent), _d(W), _d(w))
    return w


def forces(m, r, parent, level, X, n_d=2, G=1.0):
    m = _f64(m); r = _f64(r, (-1, 3)); X = _f64(X, (-1, 3))
    parent = np.ascontiguousarray(parent, np.int32); level = np.ascontiguousarray(level, np.int32)
    a = np.empty_like(r); U = C.c_double()
    lib().orc_forces(len(m), _d(m), G, _i(parent), _i(level), int(n_d), _d(r), _d(X), _d(a), C.byref(U))
    return a, U.value


def neville(nseq, S):
    nseq = np.ascontiguousarray(nseq, np.int32); S = _f64(S); kf, nvar = S.shape
    Tkk = np.empty(nvar); Tprev = np.empty(nvar)
    lib().orc_neville(kf, _i(nseq), nvar, _d(S), _d(Tkk), _d(Tprev))
    return Tkk, Tprev


def gbs_error(parent, Tkk, Tprev, X0, V0, A0, t0, T0, B, U0, H, k_fix=8) -> float:
    """Eq. gbs-criterion (orc_gbs_error): Tkk, Tprev of length 6n+1; X0, V0, A0 edge vectors n x 3."""
    parent = np.ascontiguousarray(parent, np.int32)
    n = len(parent)
    Tkk = _f64(Tkk); Tprev = _f64(Tprev)
    X0 = _f64(X0, (-1, 3)); V0 = _f64(V0, (-1, 3)); A0 = _f64(A0, (-1, 3))
    assert Tkk.shape == (6 * n + 1,) and Tprev.shape == (6 * n + 1,) and X0.shape == (n, 3)
    return lib().orc_gbs_error(n, _i(parent), _d(Tkk), _d(Tprev), _d(X0), _d(V0), _d(A0), float(t0), float(T0),
                               float(B), float(U0), float(H), int(k_fix))


def div_assign(k_fix, n_div):
    g = np.empty(k_fix, np.int32)
    mx = lib().orc_div_assign(int(k_fix), int(n_div), _i(g))
    return mx, g


def gbs_harmonic(w, x0, p0, H, k_fix=8):
    out = np.empty(2); prev = np.empty(2)
    lib().orc_gbs_harmonic(w, x0, p0, H, int(k_fix), _d(out), _d(prev))
    return out, prev


class System:
    """An N-body system integrated by the oracle."""

    def __init__(self, m, r, v, params: Params | None = None, **kw):
        self.p = params if params is not None else default_params(**kw)
        m = _f64(m); r = _f64(r, (-1, 3)); v = _f64(v, (-1, 3))
        self.n = len(m)
        self._h = lib().orc_create(self.n, _d(m), _d(r), _d(v), C.byref(self.p))
        if not self._h:
            raise ValueError("invalid system for the oracle")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_free(h)
            self._h = None

    def state(self):
        t = C.c_double(); H = C.c_double(); B = C.c_double()
        r = np.empty((self.n, 3)); v = np.empty((self.n, 3))
        lib().orc_get_state(self._h, C.byref(t), _d(r), _d(v), C.byref(H), C.byref(B))
        return dict(t=t.value, r=r, v=v, H=H.value, B=B.value)

    def set_H(self, H):
        lib().orc_set_H(self._h, float(H))

    def attempt(self, H):
        eps = C.c_double(); t = C.c_double(); U0 = C.c_double()
        r = np.empty((self.n, 3)); v = np.empty((self.n, 3))
        lib().orc_attempt(self._h, float(H), C.byref(eps), _d(r), _d(v), C.byref(t), C.byref(U0))
        return dict(eps=eps.value, r=r, v=v, t=t.value, U0=U0.value)

    def leapfrog(self, nsub, H):
        t = C.c_double(); r = np.empty((self.n, 3)); v = np.empty((self.n, 3))
        lib().orc_leapfrog(self._h, int(nsub), float(H), _d(r), _d(v), C.byref(t))
        return dict(r=r, v=v, t=t.value)

    def set_state(self, t, r, v):
        r = _f64(r, (-1, 3)); v = _f64(v, (-1, 3))
        lib().orc_set_state(self._h, float(t), _d(r), _d(v))

    def integrate(self, t_end, max_steps=1 << 30):
        st = Stats()
        rc = lib().orc_integrate(self._h, float(t_end), int(max_steps), C.byref(st))
        return rc, dict(accepted=st.accepted, rejected=st.rejected, force_evals=st.force_evals,
                        time_iters=st.time_iters, eps_last=st.eps_last, H=st.H, t=st.t)

    def energy(self):
        E = C.c_double(); T = C.c_double(); U = C.c_double(); P = np.empty(3); L = np.empty(3)
        lib().orc_energy(self._h, C.byref(E), C.byref(T), C.byref(U), _d(P), _d(L))
        return dict(E=E.value, T=T.value, U=U.value, P=P, L=L)

    def fixed_run(self, H, nsteps):
        """nsteps GBS steps of fixed fictitious step H, every attempt accepted."""
        lib().orc_fixed_run(self._h, float(H), int(nsteps))


def fixed_run_tl(m, r, v, dm, dr, dv, H, nsteps, params: Params | None = None, **kw):
    """Tangent-linear of the fixed-step run from the raw inputs (m, r, v) along (dm, dr, dv):
    dict(r, v, E) of the final state and their directional derivatives dr, dv, dE."""
    p = params if params is not None else default_params(**kw)
    m = _f64(m); n = len(m)
    r = _f64(r, (n, 3)); v = _f64(v, (n, 3))
    dm = _f64(dm); dr = _f64(dr, (n, 3)); dv = _f64(dv, (n, 3))
    rf = np.empty((n, 3)); vf = np.empty((n, 3)); drf = np.empty((n, 3)); dvf = np.empty((n, 3))
    E = C.c_double(); dE = C.c_double()
    rc = lib().orc_fixed_run_tl(n, _d(m), _d(r), _d(v), _d(dm), _d(dr), _d(dv), C.byref(p), float(H), int(nsteps),
                                _d(rf), _d(vf), C.byref(E), _d(drf), _d(dvf), C.byref(dE))
    if rc != 0:
        raise ValueError(f"orc_fixed_run_tl failed ({rc})")
    return dict(r=rf, v=vf, E=E.value, dr=drf, dv=dvf, dE=dE.value)
