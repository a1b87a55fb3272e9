"""Seeded synthetic initial conditions (inputs only; none of the integrator's arithmetic).

Both the CUDA path and the CPU oracle consume what this module produces, so it holds
no step of the method: only random draws, the Plummer-sphere sampling recipe, Kepler
orbital elements turned into state vectors, and the frame shift that makes a sample
start at rest at the origin.

Random numbers: SplitMix64 (Steele, Lea & Flood 2014) used as a counter-based
generator: draw i of stream (seed, s) is mix64(key(seed, s) + (i + 1) * gamma). The
stream is therefore reproducible on any machine and any numpy version.

Units: N-body units, G = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (finaliser) on a uint64 array."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based uniform stream keyed by (seed, stream id)."""

    def __init__(self, seed: int, stream: int = 0):
        with np.errstate(over="ignore"):
            k = np.array([(seed * 0x2545F4914F6CDD1D + stream * 0x9E3779B97F4A7C15 + 1) % (1 << 64)],
                         dtype=np.uint64)
        self._key = _mix64(k)[0]
        self._ctr = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self._ctr + 1, self._ctr + n + 1, dtype=np.uint64)
        self._ctr += n
        with np.errstate(over="ignore"):
            return _mix64(self._key + idx * _GAMMA)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) with 53 random bits each."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def uniform1(self) -> float:
        return float(self.uniform(1)[0])


def _to_rest_frame(m, r, v):
    mt = m.sum()
    r = r - (m[:, None] * r).sum(axis=0) / mt
    v = v - (m[:, None] * v).sum(axis=0) / mt
    return r, v


def _isotropic(st: Stream, n: int) -> np.ndarray:
    u = st.uniform(n)
    w = st.uniform(n)
    cz = 1.0 - 2.0 * u
    sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
    ph = 2.0 * math.pi * w
    return np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=1)


def plummer(n: int, seed: int, total_mass: float = 1.0, r_cut_virial: float = 10.0):
    """Equal-mass Plummer sphere, virial radius 1, sampled as in Aarseth, Henon & Wielen (1974).

    Radius from the enclosed-mass fraction, speed by rejection from
    g(q) = q^2 (1 - q^2)^(7/2), isotropic directions; radii beyond r_cut_virial virial
    radii are redrawn. Returns (m, r, v) with r, v of shape (n, 3), at rest at the origin.
    """
    st = Stream(seed, 1)
    # Henon units (G = M = a = 1) first; virial radius there is 16 / (3 pi).
    rcut = r_cut_virial * 16.0 / (3.0 * math.pi)
    rad = np.empty(n)
    filled = 0
    while filled < n:
        x = st.uniform(n - filled)
        x = np.where(x <= 0.0, 1e-300, x)
        rr = 1.0 / np.sqrt(np.power(x, -2.0 / 3.0) - 1.0)
        ok = rr[rr <= rcut]
        rad[filled:filled + ok.size] = ok
        filled += ok.size
    pos = rad[:, None] * _isotropic(st, n)
    q = np.empty(n)
    filled = 0
    while filled < n:
        k = max(4 * (n - filled), 16)
        x4 = st.uniform(k)
        x5 = st.uniform(k)
        acc = x4[0.1 * x5 < x4 * x4 * np.power(1.0 - x4 * x4, 3.5)]
        take = acc[: n - filled]
        q[filled:filled + take.size] = take
        filled += take.size
    speed = q * math.sqrt(2.0) * np.power(1.0 + rad * rad, -0.25)
    vel = speed[:, None] * _isotropic(st, n)
    a = 3.0 * math.pi / 16.0
    pos = pos * a
    vel = vel / math.sqrt(a)
    if total_mass != 1.0:
        vel = vel * math.sqrt(total_mass)
    m = np.full(n, total_mass / n)
    pos, vel = _to_rest_frame(m, pos, vel)
    return m, pos, vel


def hernquist_df(binding, G=1.0, M=1.0, a=1.0):
    """Isotropic distribution function f(E) of the Hernquist (1990) sphere, the closed form
    of Eddington's inversion, for binding energy per unit mass E = Psi - v^2/2 in
    [0, GM/a): with q = sqrt(a E / (G M)) and v_g = sqrt(G M / a),
    f = M / (8 sqrt(2) pi^3 a^3 v_g^3) (1 - q^2)^(-5/2)
        [3 asin q + q sqrt(1 - q^2) (1 - 2 q^2) (8 q^4 - 8 q^2 - 3)]."""
    q = np.sqrt(np.clip(a * np.asarray(binding, np.float64) / (G * M), 0.0, 1.0 - 1e-16))
    vg = math.sqrt(G * M / a)
    q2 = q * q
    br = 3.0 * np.arcsin(q) + q * np.sqrt(1.0 - q2) * (1.0 - 2.0 * q2) * (8.0 * q2 * q2 - 8.0 * q2 - 3.0)
    return M / (8.0 * math.sqrt(2.0) * math.pi ** 3 * a ** 3 * vg ** 3) * np.power(1.0 - q2, -2.5) * np.maximum(br, 0.0)


def hernquist(n: int, seed: int, total_mass: float = 1.0, r_half: float = 1.0, r_cut_half: float = 20.0,
              reject_hard_binaries: bool = True, max_draws: int = 1000):
    """Equal-mass Hernquist sphere (Sec. 6.1): density M a / (2 pi r (r + a)^3) with
    a = r_half / (1 + sqrt 2), so that half the mass lies inside r_half. Radii from the
    enclosed-mass fraction M(<r)/M = (r / (r + a))^2 (redrawn beyond r_cut_half half-mass
    radii); speeds by rejection from v^2 f(Psi(r) - v^2/2), f the isotropic distribution
    function (Eddington's formula, closed form), Psi = G M / (r + a); isotropic directions;
    G = 1; shifted to rest at the origin.

    A cluster that holds a hard binary is drawn again (the next draw of the same stream): a
    pair is hard when its two-body binding energy G m_i m_j / (2 a_ij) exceeds the mean
    kinetic energy of a particle, m sigma^2 / 2 with sigma^2 = sum m v^2 / sum m.
    Returns (m, r, v, draws)."""
    st = Stream(seed, 31)
    a = r_half / (1.0 + math.sqrt(2.0))
    rcut = r_cut_half * r_half
    for draw in range(1, max_draws + 1):
        rad = np.empty(n)
        filled = 0
        while filled < n:
            x = st.uniform(n - filled)
            s = np.sqrt(x)
            with np.errstate(divide="ignore"):
                rr = a * s / (1.0 - s)
            ok = rr[(rr <= rcut) & np.isfinite(rr)]
            rad[filled:filled + ok.size] = ok
            filled += ok.size
        pos = rad[:, None] * _isotropic(st, n)
        psi = total_mass / (rad + a)
        vesc = np.sqrt(2.0 * psi)
        grid = np.linspace(0.0, 1.0, 257)[1:-1]
        speed = np.empty(n)
        for i in range(n):
            vv = grid * vesc[i]
            gmax = 1.05 * float(np.max(vv * vv * hernquist_df(psi[i] - 0.5 * vv * vv, M=total_mass, a=a)))
            while True:
                u1, u2 = st.uniform(2)
                v = u1 * vesc[i]
                if u2 * gmax <= v * v * float(hernquist_df(psi[i] - 0.5 * v * v, M=total_mass, a=a)):
                    speed[i] = v
                    break
        vel = speed[:, None] * _isotropic(st, n)
        m = np.full(n, total_mass / n)
        pos, vel = _to_rest_frame(m, pos, vel)
        if not reject_hard_binaries or not has_hard_binary(m, pos, vel):
            return m, pos, vel, draw
    raise RuntimeError("no Hernquist sample without a hard binary")


def has_hard_binary(m, r, v, G=1.0):
    """True if some pair's two-body binding energy exceeds m sigma^2 / 2 (Sec. 6.1)."""
    m = np.asarray(m, np.float64)
    sigma2 = float((m * (v * v).sum(axis=1)).sum() / m.sum())
    threshold = 0.5 * float(m.mean()) * sigma2
    d = r[:, None, :] - r[None, :, :]
    dv = v[:, None, :] - v[None, :, :]
    dist = np.sqrt((d * d).sum(axis=2))
    mu = m[:, None] * m[None, :] / (m[:, None] + m[None, :])
    with np.errstate(divide="ignore"):
        e_rel = 0.5 * mu * (dv * dv).sum(axis=2) - G * m[:, None] * m[None, :] / dist
    iu = np.triu_indices(len(m), 1)
    return bool(np.any(e_rel[iu] < -threshold))


def random_rotation(st: Stream) -> np.ndarray:
    """Uniform random rotation matrix from a unit quaternion (Shoemake 1992)."""
    u1, u2, u3 = st.uniform(3)
    a = math.sqrt(1 - u1)
    b = math.sqrt(u1)
    qx, qy, qz, qw = (a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2),
                      b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3))
    return np.array([
        [1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
        [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
        [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)],
    ])


def kepler_state(m1: float, m2: float, a: float, e: float, true_anomaly: float = 0.0,
                 inc: float = 0.0, node: float = 0.0, peri: float = 0.0):
    """Relative position/velocity (r2 - r1, v2 - v1) of a Kepler orbit with G = 1."""
    mu = m1 + m2
    p = a * (1.0 - e * e)
    f = true_anomaly
    rr = p / (1.0 + e * math.cos(f))
    x = np.array([rr * math.cos(f), rr * math.sin(f), 0.0])
    h = math.sqrt(mu * p)
    v = np.array([-mu / h * math.sin(f), mu / h * (e + math.cos(f)), 0.0])
    # rotation: R_z(node) R_x(inc) R_z(peri)
    cO, sO, ci, si, cw, sw = (math.cos(node), math.sin(node), math.cos(inc), math.sin(inc),
                              math.cos(peri), math.sin(peri))
    R = np.array([
        [cO * cw - sO * sw * ci, -cO * sw - sO * cw * ci, sO * si],
        [sO * cw + cO * sw * ci, -sO * sw + cO * cw * ci, -cO * si],
        [sw * si, cw * si, ci],
    ])
    return R @ x, R @ v


def kepler_binary(seed: int = 0, m1: float = 0.5, m2: float = 0.5, a: float = 1.0,
                  e: float = 0.9, true_anomaly: float = math.pi, orient: bool = True):
    """Two-body problem; by default starts at apocentre in a seeded random orientation."""
    dr, dv = kepler_state(m1, m2, a, e, true_anomaly)
    if orient:
        R = random_rotation(Stream(seed, 7))
        dr, dv = R @ dr, R @ dv
    m = np.array([m1, m2])
    r = np.stack([-m2 / (m1 + m2) * dr, m1 / (m1 + m2) * dr])
    v = np.stack([-m2 / (m1 + m2) * dv, m1 / (m1 + m2) * dv])
    return m, r, v


def pythagorean():
    """Burrau's problem: masses 3, 4, 5 at rest at the corners of a 3-4-5 right triangle,
    each body opposite the side of the same length (mass 5 at the right angle)."""
    m = np.array([3.0, 4.0, 5.0])
    r = np.array([[1.0, 3.0, 0.0], [-2.0, -1.0, 0.0], [1.0, -1.0, 0.0]])
    v = np.zeros((3, 3))
    r, v = _to_rest_frame(m, r, v)
    return m, r, v


def hierarchical_triple(m1: float, m2: float, m3: float, a_in: float, e_in: float,
                        a_out: float, e_out: float, inc: float, st: Stream | None = None):
    """Inner binary (m1, m2) plus an outer body m3; inclination between the orbital planes
    is `inc`. Phases and nodes are drawn from `st` when given, else zero."""
    if st is not None:
        f_in, f_out, node, w_in = (2 * math.pi * x for x in st.uniform(4))
    else:
        f_in = f_out = node = w_in = 0.0
    dr_in, dv_in = kepler_state(m1, m2, a_in, e_in, f_in, inc=inc, node=node, peri=w_in)
    dr_out, dv_out = kepler_state(m1 + m2, m3, a_out, e_out, f_out)
    mb = m1 + m2
    r1 = -m2 / mb * dr_in
    r2 = m1 / mb * dr_in
    v1 = -m2 / mb * dv_in
    v2 = m1 / mb * dv_in
    mt = mb + m3
    rb = -m3 / mt * dr_out
    vb = -m3 / mt * dv_out
    r3 = mb / mt * dr_out
    v3 = mb / mt * dv_out
    m = np.array([m1, m2, m3])
    r = np.stack([r1 + rb, r2 + rb, r3])
    v = np.stack([v1 + vb, v2 + vb, v3])
    r, v = _to_rest_frame(m, r, v)
    return m, r, v


def lidov_kozai():
    """Primary 1, secondary 1e-6 (test particle), perturber 1 (the paper's 1e9, 1e3, 1e9
    solar masses scaled by 1e9): inner a=2, e=1e-3; outer a=20, e=0; inclination 80 deg."""
    return hierarchical_triple(1.0, 1e-6, 1.0, 2.0, 1e-3, 20.0, 0.0, math.radians(80.0))


def plummer_smbh_binary(n_stars: int = 2048, seed: int = 2, m_bh: float = 0.01, a_bh: float = 0.01):
    """Plummer sphere (stellar mass 1) plus a central circular SMBH binary of two masses m_bh
    with separation a_bh, in a seeded random orientation. N = n_stars + 2."""
    m, r, v = plummer(n_stars, seed)
    R = random_rotation(Stream(seed, 11))
    vrel = math.sqrt(2.0 * m_bh / a_bh)
    dr = R @ np.array([a_bh, 0.0, 0.0])
    dv = R @ np.array([0.0, vrel, 0.0])
    mb = np.array([m_bh, m_bh])
    rb = np.stack([-0.5 * dr, 0.5 * dr])
    vb = np.stack([-0.5 * dv, 0.5 * dv])
    m = np.concatenate([m, mb])
    r = np.concatenate([r, rb])
    v = np.concatenate([v, vb])
    r, v = _to_rest_frame(m, r, v)
    return m, r, v


def plummer_two_smbh(n_stars: int = 10000, seed: int = 5, m_bh: float = 0.005, d: float = 0.1):
    """Plummer sphere (stellar mass 1) plus two SMBHs of mass m_bh at +/- d on the x axis,
    moving at +/- half the local circular speed along y. The circular speed counts the
    Plummer mass inside d and the pull of the other hole: v_c^2 = d (M(<d)/d^2 + m_bh/(2d)^2)."""
    m, r, v = plummer(n_stars, seed)
    a = 3.0 * math.pi / 16.0
    m_in = d ** 3 / (d * d + a * a) ** 1.5
    vc = math.sqrt(d * (m_in / (d * d) + m_bh / (2 * d) ** 2))
    rb = np.array([[d, 0.0, 0.0], [-d, 0.0, 0.0]])
    vb = np.array([[0.0, 0.5 * vc, 0.0], [0.0, -0.5 * vc, 0.0]])
    m = np.concatenate([m, [m_bh, m_bh]])
    r = np.concatenate([r, rb])
    v = np.concatenate([v, vb])
    r, v = _to_rest_frame(m, r, v)
    return m, r, v


def perturbed(m, r, v, realisation: int, rel: float = 1e-15):
    """Realisation `realisation` of an ensemble around (m, r, v): 0 is the input itself;
    k > 0 multiplies every position and velocity component by 1 + rel (2u - 1), u uniform
    from stream (7919, k). A rounding-level change of the start, so that the runs of an
    ensemble sample the spread of rounding and truncation along their step sequences."""
    if realisation == 0:
        return m, r.copy(), v.copy()
    st = Stream(7919, realisation)
    n = len(m)
    fr = 1.0 + rel * (2.0 * st.uniform(3 * n) - 1.0)
    fv = 1.0 + rel * (2.0 * st.uniform(3 * n) - 1.0)
    return m, r * fr.reshape(n, 3), v * fv.reshape(n, 3)


@dataclass
class System:
    m: np.ndarray
    r: np.ndarray
    v: np.ndarray


def batched_systems(count: int = 4096, seed: int = 3, n_min: int = 3, n_max: int = 200):
    """Independent subsystems of uneven sizes. Even indices: hierarchical triples (masses
    1, 1, 0.1; inner a=1, e~U[0,0.9]; outer a~U[10,50], e=0; inclination ~U[40,140] deg).
    Odd indices: Plummer clusters of N_i = round(exp U[ln n_min, ln n_max]) bodies, N_i - 1
    equal-mass stars plus a central point mass of 0.1 of the stellar mass."""
    st = Stream(seed, 21)
    out = []
    for i in range(count):
        if i % 2 == 0:
            e_in, a_out, inc = st.uniform(3)
            m, r, v = hierarchical_triple(1.0, 1.0, 0.1, 1.0, 0.9 * e_in, 10.0 + 40.0 * a_out, 0.0,
                                          math.radians(40.0 + 100.0 * inc), st)
        else:
            x = st.uniform1()
            n_i = int(round(math.exp(math.log(n_min) + x * (math.log(n_max) - math.log(n_min)))))
            n_i = max(n_i, 3)
            ms, rs, vs = plummer(n_i - 1, seed * 100003 + i)
            m = np.concatenate([ms, [0.1 * ms.sum()]])
            r = np.concatenate([rs, np.zeros((1, 3))])
            v = np.concatenate([vs, np.zeros((1, 3))])
            r, v = _to_rest_frame(m, r, v)
        out.append(System(m, r, v))
    return out


# The workloads the tests and the benchmark use, by name.
def workload(name: str):
    if name == "plummer64":
        return plummer(64, 1)
    if name == "plummer2048_smbh_binary":
        return plummer_smbh_binary(2048, 2)
    if name == "plummer256":
        return plummer(256, 4)
    if name == "plummer10k_two_smbh":
        return plummer_two_smbh(10000, 5)
    if name.startswith("hernquist379_seed"):
        return hernquist(379, int(name[len("hernquist379_seed"):]))[:3]
    raise KeyError(name)
