"""Python access to the FP64 CPU oracle in ``dbm_oracle.c``.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this module; the product path never
does.  It compiles the C oracle with gcc (``-O2 -ffp-contract=off
-fopenmp``), loads it with ctypes and wraps each routine for numpy arrays.

Every wrapped routine restates a passage of arXiv 2006.15932 (Lin, Luo, Fei
& Succi); the C file names the passage beside each routine.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dbm_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")

Q = 16
MAXS = 8
PERIODIC, OUTFLOW = 0, 1

STATUS_BITS = {1: "bad density", 2: "bad temperature", 4: "negative n*", 8: "non-finite f"}


class _Species(C.Structure):
    _fields_ = [
        ("m", C.c_double),
        ("I", C.c_double),
        ("tau", C.c_double),
        ("v", C.c_double * 4),
        ("eta", C.c_double * 4),
        ("a", C.c_double),
    ]


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int),
        ("ny", C.c_int),
        ("ns", C.c_int),
        ("dx", C.c_double),
        ("dy", C.c_double),
        ("dt", C.c_double),
        ("bc_x", C.c_int),
        ("bc_y", C.c_int),
        ("fuel", C.c_int),
        ("oxid", C.c_int),
        ("k_ov", C.c_double),
        ("Ea_over_R", C.c_double),
        ("Q", C.c_double),
        ("ax", C.c_double),
        ("ay", C.c_double),
        ("sp", _Species * MAXS),
    ]


@dataclass
class Species:
    """Per-species constants: molar mass m, extra degrees of freedom I,
    relaxation time tau, ring speeds v_a..v_d, internal speeds eta_a..eta_d
    and stoichiometric coefficient a."""

    m: float = 1.0
    I: float = 3.0
    tau: float = 2e-5
    v: Sequence[float] = (1.3, 1.2, 2.9, 2.4)
    eta: Sequence[float] = (2.2, 0.7, 0.4, 0.3)
    a: float = 0.0


@dataclass
class Params:
    nx: int
    ny: int
    species: list
    dx: float = 1e-3
    dy: float = 1e-3
    dt: float = 1e-5
    bc_x: int = PERIODIC
    bc_y: int = PERIODIC
    fuel: int = 0
    oxid: int = 1
    k_ov: float = 0.0
    Ea_over_R: float = 0.0
    Q: float = 0.0
    accel: tuple = (0.0, 0.0)

    @property
    def ns(self) -> int:
        return len(self.species)

    def to_c(self) -> _Params:
        p = _Params()
        p.nx, p.ny, p.ns = self.nx, self.ny, self.ns
        p.dx, p.dy, p.dt = self.dx, self.dy, self.dt
        p.bc_x, p.bc_y = self.bc_x, self.bc_y
        p.fuel, p.oxid = self.fuel, self.oxid
        p.k_ov, p.Ea_over_R, p.Q = self.k_ov, self.Ea_over_R, self.Q
        p.ax, p.ay = float(self.accel[0]), float(self.accel[1])
        for s, sp in enumerate(self.species):
            c = p.sp[s]
            c.m, c.I, c.tau, c.a = sp.m, sp.I, sp.tau, sp.a
            for r in range(4):
                c.v[r] = sp.v[r]
                c.eta[r] = sp.eta[r]
        return p


def params_of(problem) -> Params:
    """The oracle's parameter record for a problem description: any object
    with the attributes nx, ny, species (each with m, I, tau, v, eta, a), dx,
    dy, dt, bc_x, bc_y, fuel, oxid, k_ov, Ea_over_R, Q and accel, such as the
    seeded workloads of the test inputs.  Reads attributes only."""
    pb = problem
    sp = [Species(m=s.m, I=s.I, tau=s.tau, v=tuple(s.v), eta=tuple(s.eta), a=s.a) for s in pb.species]
    return Params(nx=pb.nx, ny=pb.ny, species=sp, dx=pb.dx, dy=pb.dy, dt=pb.dt, bc_x=pb.bc_x,
                  bc_y=pb.bc_y, fuel=pb.fuel, oxid=pb.oxid, k_ov=pb.k_ov, Ea_over_R=pb.Ea_over_R,
                  Q=pb.Q, accel=tuple(pb.accel))


_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so``."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC)):
        return LIB_PATH
    tmp = LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB_PATH)
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(_Params)
        L.orc_moment_matrix.argtypes = [dp, dp, dp, dp]
        L.orc_velocities.argtypes = [C.POINTER(_Species), dp, dp, dp]
        L.orc_invert.argtypes = [dp, dp, C.c_int]
        L.orc_invert.restype = C.c_int
        L.orc_fhat.argtypes = [C.c_double] * 6 + [dp]
        L.orc_prepare.argtypes = [pp, dp]
        L.orc_prepare.restype = C.c_int
        L.orc_cell_rhs.argtypes = [pp, dp, dp, dp]
        L.orc_cell_rhs.restype = C.c_int
        L.orc_species_moments.argtypes = [dp, dp, dp, dp, C.c_double, C.c_double] + [dp] * 5
        L.orc_mixture.argtypes = [C.c_int, C.POINTER(_Species), dp, dp, dp, dp, dp, dp, dp]
        L.orc_omega.argtypes = [pp, dp, C.c_double]
        L.orc_omega.restype = C.c_double
        L.orc_dTdt.argtypes = [pp, dp, C.c_double, C.c_double]
        L.orc_dTdt.restype = C.c_double
        L.orc_minmod.argtypes = [C.c_double, C.c_double]
        L.orc_minmod.restype = C.c_double
        L.orc_nnd_dflux.argtypes = [C.c_double, dp, C.c_double]
        L.orc_nnd_dflux.restype = C.c_double
        L.orc_step_region.argtypes = [pp, dp, dp, dp] + [C.c_int] * 4
        L.orc_step_region.restype = C.c_int
        L.orc_run.argtypes = [pp, dp, dp, C.c_int]
        L.orc_run.restype = C.c_int
        L.orc_init_feq.argtypes = [pp, dp, dp, dp, dp, dp]
        L.orc_init_feq.restype = C.c_int
        L.orc_moments.argtypes = [pp, dp, dp]
        L.orc_nonequilibrium.argtypes = [pp, dp, dp]
        L.orc_conservation.argtypes = [pp, dp, dp]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = C.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "need C-contiguous float64"
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------------------
# velocity space and equilibrium
# ---------------------------------------------------------------------------

def velocities(sp: Species):
    """(vx, vy, eta), 16 each, of the D2V16 set of one species."""
    c = _Species()
    c.m, c.I, c.tau, c.a = sp.m, sp.I, sp.tau, sp.a
    for r in range(4):
        c.v[r], c.eta[r] = sp.v[r], sp.eta[r]
    vx, vy, eta = (np.zeros(Q) for _ in range(3))
    lib().orc_velocities(C.byref(c), _dp(vx), _dp(vy), _dp(eta))
    return vx, vy, eta


def moment_matrix(sp: Species) -> np.ndarray:
    vx, vy, eta = velocities(sp)
    M = np.zeros((Q, Q))
    lib().orc_moment_matrix(_dp(vx), _dp(vy), _dp(eta), _dp(M))
    return M


def invert(A) -> np.ndarray:
    A = _f64(A)
    n = A.shape[0]
    out = np.zeros_like(A)
    if lib().orc_invert(_dp(A), _dp(out), n) != 0:
        raise np.linalg.LinAlgError("singular matrix")
    return out


def minv(params: Params) -> np.ndarray:
    """S x 16 x 16 blocks of M^-1."""
    out = np.zeros((params.ns, Q, Q))
    cp = params.to_c()
    if lib().orc_prepare(C.byref(cp), _dp(out)) != 0:
        raise np.linalg.LinAlgError("singular moment matrix")
    return out


def fhat(n, ux, uy, T, m, I) -> np.ndarray:
    out = np.zeros(Q)
    lib().orc_fhat(n, ux, uy, T, m, I, _dp(out))
    return out


def feq(sp: Species, n, ux, uy, T) -> np.ndarray:
    M = moment_matrix(sp)
    return invert(M) @ fhat(n, ux, uy, T, sp.m, sp.I)


# ---------------------------------------------------------------------------
# one cell
# ---------------------------------------------------------------------------

def cell_rhs(params: Params, fc) -> tuple[np.ndarray, int]:
    """Omega + R + G for the S x 16 distributions of one cell."""
    fc = _f64(fc).reshape(params.ns, Q)
    Mi = minv(params)
    out = np.zeros_like(fc)
    cp = params.to_c()
    st = lib().orc_cell_rhs(C.byref(cp), _dp(Mi), _dp(fc), _dp(out))
    return out, st


def species_moments(sp: Species, f):
    vx, vy, eta = velocities(sp)
    f = _f64(f)
    vals = [C.c_double() for _ in range(5)]
    lib().orc_species_moments(_dp(f), _dp(vx), _dp(vy), _dp(eta), sp.m, sp.I,
                              *[C.byref(v) for v in vals])
    return tuple(v.value for v in vals)  # n, ux, uy, T^s, E


def mixture(params: Params, n, ux, uy, E):
    cp = params.to_c()
    n, ux, uy, E = (_f64(a) for a in (n, ux, uy, E))
    out = [C.c_double() for _ in range(3)]
    lib().orc_mixture(params.ns, cp.sp, _dp(n), _dp(ux), _dp(uy), _dp(E),
                      *[C.byref(v) for v in out])
    return tuple(v.value for v in out)


def omega(params: Params, n, T) -> float:
    cp = params.to_c()
    return lib().orc_omega(C.byref(cp), _dp(_f64(n)), T)


def dTdt(params: Params, n, T, w) -> float:
    cp = params.to_c()
    return lib().orc_dTdt(C.byref(cp), _dp(_f64(n)), T, w)


def minmod(a, b) -> float:
    return lib().orc_minmod(a, b)


def nnd_dflux(c, w5, h) -> float:
    return lib().orc_nnd_dflux(c, _dp(_f64(w5)), h)


# ---------------------------------------------------------------------------
# grid
# ---------------------------------------------------------------------------

def init_feq(params: Params, rho_s, ux, uy, T) -> np.ndarray:
    """f[s][i][y][x] = f^eq(rho^s/m^s, u, T); inputs are [s][y][x] / [y][x]."""
    shape = (params.ny, params.nx)
    rho_s = _f64(rho_s).reshape(params.ns, *shape)
    ux, uy, T = (_f64(a).reshape(shape) for a in (ux, uy, T))
    f = np.zeros((params.ns, Q) + shape)
    cp = params.to_c()
    if lib().orc_init_feq(C.byref(cp), _dp(rho_s), _dp(ux), _dp(uy), _dp(T), _dp(f)) != 0:
        raise np.linalg.LinAlgError("singular moment matrix")
    return f


def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP loops (n > 0 sets them; timing only);
    returns the number in use."""
    return int(lib().orc_set_threads(int(n)))


def run(params: Params, f, nsteps: int) -> tuple[np.ndarray, int]:
    """nsteps forward-Euler steps of the whole grid; returns (f, status)."""
    f = _f64(f).reshape(params.ns, Q, params.ny, params.nx).copy()
    work = np.empty_like(f)
    cp = params.to_c()
    st = lib().orc_run(C.byref(cp), _dp(f), _dp(work), int(nsteps))
    if st < 0:
        raise np.linalg.LinAlgError("singular moment matrix")
    return f, st


def step_region(params: Params, f, x0, x1, y0, y1) -> tuple[np.ndarray, int]:
    """One step of the cells [x0,x1) x [y0,y1) from the full field f; the
    returned array holds only that region, shape (S, 16, y1-y0, x1-x0)."""
    f = _f64(f).reshape(params.ns, Q, params.ny, params.nx)
    out = np.zeros((params.ns, Q, y1 - y0, x1 - x0))
    Mi = minv(params)
    cp = params.to_c()
    st = lib().orc_step_region(C.byref(cp), _dp(Mi), _dp(f), _dp(out), x0, x1, y0, y1)
    return out, st


def moments(params: Params, f) -> np.ndarray:
    f = _f64(f).reshape(params.ns, Q, params.ny, params.nx)
    out = np.zeros((4 * params.ns + 5, params.ny, params.nx))
    cp = params.to_c()
    lib().orc_moments(C.byref(cp), _dp(f), _dp(out))
    return out


def nonequilibrium(params: Params, f) -> np.ndarray:
    f = _f64(f).reshape(params.ns, Q, params.ny, params.nx)
    out = np.zeros((20 * params.ns, params.ny, params.nx))
    cp = params.to_c()
    lib().orc_nonequilibrium(C.byref(cp), _dp(f), _dp(out))
    return out


def conservation(params: Params, f) -> np.ndarray:
    f = _f64(f).reshape(params.ns, Q, params.ny, params.nx)
    out = np.zeros(params.ns + 4)
    cp = params.to_c()
    lib().orc_conservation(C.byref(cp), _dp(f), _dp(out))
    return out
