"""Seeded synthetic inputs shared by the tests, the smoke check and the
benchmark.

This module holds problem descriptions (grid, species constants, reaction
and force parameters) and macroscopic initial fields (rho^s, u, T).  It does
none of the method's arithmetic: the distributions themselves are built by
whoever consumes a problem (the CUDA library through ``dbm_set_state``, the
oracle through its own equilibrium routine).

Units are nondimensional: m = 1, T = 1 and unit density give a thermal speed
of order one.  D2V16 ring speeds and internal speeds default to
(1.3, 1.2, 2.9, 2.4; 2.2, 0.7, 0.4, 0.3) * sqrt(T_ref / m), which follows the
paper's guidance (section "Numerical simulation") of placing v near
sqrt(D T/m) and |u| and eta near sqrt(I T/m); its moment matrix has a
condition number of about 4e2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Sequence

import numpy as np

PERIODIC, OUTFLOW = 0, 1
SEED = 20200627

DEFAULT_V = (1.3, 1.2, 2.9, 2.4)
DEFAULT_ETA = (2.2, 0.7, 0.4, 0.3)


@dataclass
class SpeciesSpec:
    m: float = 1.0
    I: float = 3.0
    tau: float = 2e-5
    v: Sequence[float] = DEFAULT_V
    eta: Sequence[float] = DEFAULT_ETA
    a: float = 0.0


def species(m=1.0, I=3.0, tau=2e-5, a=0.0, T_ref=1.0, v=DEFAULT_V, eta=DEFAULT_ETA) -> SpeciesSpec:
    s = math.sqrt(T_ref / m)
    return SpeciesSpec(m=m, I=I, tau=tau, v=tuple(x * s for x in v), eta=tuple(x * s for x in eta), a=a)


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    species: List[SpeciesSpec]
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
    nsteps: int = 1
    # macroscopic initial fields: rho_s (S, ny, nx), ux/uy/T (ny, nx)
    rho_s: np.ndarray = None
    ux: np.ndarray = None
    uy: np.ndarray = None
    T: np.ndarray = None

    @property
    def ns(self) -> int:
        return len(self.species)

    @property
    def cells(self) -> int:
        return self.nx * self.ny


# ---------------------------------------------------------------------------
# configurations
# ---------------------------------------------------------------------------

def sod_tube(nx: int = 400, nsteps: int = 2000) -> Problem:
    """Sod-type shock tube, two non-reacting species with mass fractions
    0.5/0.5 (m = 1, I = 3, so gamma = 1.4): rho = 1, p = 1 for x < 0.2,
    rho = 0.125, p = 0.1 beyond, u = 0; dx = 1e-3 (for 400 cells), dt = 1e-5,
    tau = 2e-5; outflow in x, periodic in y with one row."""
    L = 0.4
    dx = L / nx
    x = (np.arange(nx) + 0.5) * dx
    left = x < 0.2
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    sp = [species(m=1.0, I=3.0, tau=2e-5), species(m=1.0, I=3.0, tau=2e-5)]
    n = rho / 1.0
    T = p / n
    rho_s = np.stack([0.5 * rho, 0.5 * rho])[:, None, :]
    return Problem(name="sod_400x1_s2", nx=nx, ny=1, species=sp, dx=dx, dy=dx, dt=1e-5 * dx / 1e-3,
                   bc_x=OUTFLOW, bc_y=PERIODIC, nsteps=nsteps, rho_s=rho_s,
                   ux=np.zeros((1, nx)), uy=np.zeros((1, nx)), T=T[None, :])


def random_smooth(nx: int, ny: int, ns: int, seed: int = SEED, *, reactive: bool = False,
                  force: bool = False, bc=(PERIODIC, PERIODIC), amp: float = 0.05,
                  unequal: bool = True, dt: float = 1e-5, tau: float = 2e-5) -> Problem:
    """A smooth random state of ns species on an nx x ny grid: a few random
    Fourier modes of amplitude ``amp`` on density, velocity and temperature
    around rho^s = 1/ns, u = (0.1, -0.05), T = 1.  Unequal masses and
    relaxation times when ``unequal``.  With ``reactive`` species 0 is the
    fuel, 1 the oxidiser and the rest products (a = -1, -1, +2/(ns-2)...,
    chosen with equal masses so that sum a m = 0)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(ny) / max(ny, 1), np.arange(nx) / max(nx, 1), indexing="ij")

    def field(base, a):
        out = np.full((ny, nx), base, dtype=np.float64)
        for _ in range(3):
            kx, ky = rng.integers(1, 4, size=2)
            ph = rng.uniform(0, 2 * math.pi)
            out += a * base * rng.uniform(0.3, 1.0) * np.sin(2 * math.pi * (kx * xx + ky * yy) + ph)
        return out

    sp = []
    for s in range(ns):
        m = (1.0 + 0.5 * s) if (unequal and not reactive) else 1.0
        t = tau * ((1.0 + 0.25 * s) if unequal else 1.0)
        sp.append(species(m=m, I=3.0 + (s % 2) if unequal else 3.0, tau=t))
    if reactive:
        assert ns >= 3
        sp[0].a, sp[1].a = -1.0, -1.0
        for s in range(2, ns):
            sp[s].a = 2.0 / (ns - 2)
    rho_s = np.stack([field(1.0 / ns, amp) for _ in range(ns)])
    ux = field(0.1, amp)
    uy = field(-0.05, amp)
    T = field(1.0, amp)
    pb = Problem(name=f"random_{nx}x{ny}_s{ns}", nx=nx, ny=ny, species=sp, dx=1e-3, dy=1e-3, dt=dt,
                 bc_x=bc[0], bc_y=bc[1], rho_s=rho_s, ux=ux, uy=uy, T=T)
    if reactive:
        pb.fuel, pb.oxid = 0, 1
        pb.k_ov = 2.0e3
        pb.Ea_over_R = 2.0
        pb.Q = 1.5
    if force:
        pb.accel = (30.0, -50.0)
    return pb


def reactive_premixed(nx: int = 1024, ny: int = 256, seed: int = SEED, nsteps: int = 20000) -> Problem:
    """Premixed 2-D reactive gas, three species (fuel F, oxidiser O, product
    P), one-step reaction F + O -> 2 P (a = -1, -1, +2; m = 1 each):
    mass fractions 0.5/0.5/0 (product 1e-3 seed), rho = 1, T = 1, u = 0,
    +-1% seeded white noise on density at constant pressure; a hot product
    band at x < nx/16 ignites it.  Periodic in x and y; dx = 1e-3,
    dt = 1e-5, tau = 2e-5.  Reaction constants are drawn from a seed in
    ranges that give visible conversion within 20k steps."""
    rng = np.random.default_rng(seed)
    sp = [species(tau=2e-5, a=-1.0), species(tau=2e-5, a=-1.0), species(tau=2e-5, a=2.0)]
    noise = rng.uniform(-0.01, 0.01, size=(ny, nx))
    rho = 1.0 + noise
    T = 1.0 / rho  # constant pressure p = n T = 1
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    hot = x < nx // 16
    yF = np.where(hot, 0.05, 0.4995)
    yO = np.where(hot, 0.05, 0.4995)
    yP = 1.0 - yF - yO
    T = np.where(hot, 1.8 / rho, T)
    rho_s = np.stack([rho * yF, rho * yO, rho * yP])
    k_ov = float(rng.uniform(20.0, 40.0))
    Ea = float(rng.uniform(2.0, 3.0))
    Q = float(rng.uniform(0.6, 0.9))
    return Problem(name=f"reactive_{nx}x{ny}_s3", nx=nx, ny=ny, species=sp, dx=1e-3, dy=1e-3, dt=1e-5,
                   bc_x=PERIODIC, bc_y=PERIODIC, fuel=0, oxid=1, k_ov=k_ov, Ea_over_R=Ea, Q=Q,
                   nsteps=nsteps, rho_s=rho_s, ux=np.zeros((ny, nx)), uy=np.zeros((ny, nx)), T=T)


def premixed_flame(nx: int = 300) -> Problem:
    """A one-dimensional premixed flame (section "Flame at constant
    pressure" in spirit; the propane chemistry is not given): three species
    F + O -> 2 P (a = -1, -1, +2, m = 1), a high activation temperature
    E_a/R = 16 so that the fresh gas at T = 1 is nearly inert while the burnt
    gas at T = 1.8 reacts fast (k_ov = 1.4e6), heat Q = 8 per mole of
    reaction; burnt products (T = 1.8, 2 % reactants left) at x < 40 meet the
    fresh mixture (Y_F = Y_O = 0.5, T = 1) through a tanh profile of width
    2 cells at constant pressure p = 1; tau = 2e-4 (a thick, resolved flame),
    D2V16 ring speeds scaled for T_ref = 1.3; outflow at both ends, one row.
    The flame propagates into the fresh gas, about 0.4 cells per thousand
    steps."""
    tau = 2e-4
    sp = [species(tau=tau, a=-1.0, T_ref=1.3), species(tau=tau, a=-1.0, T_ref=1.3),
          species(tau=tau, a=2.0, T_ref=1.3)]
    x = np.arange(nx)[None, :].astype(np.float64)
    burnt = 0.5 * (1.0 - np.tanh((x - 40.0) / 2.0))
    T = 1.0 + 0.8 * burnt
    rho = 1.0 / T
    yF = 0.5 - 0.49 * burnt
    rho_s = np.stack([rho * yF, rho * yF, rho * (1.0 - 2.0 * yF)])
    return Problem(name=f"flame_{nx}", nx=nx, ny=1, species=sp, dx=1e-3, dy=1e-3, dt=1e-5, bc_x=OUTFLOW,
                   bc_y=PERIODIC, fuel=0, oxid=1, k_ov=1.4e6, Ea_over_R=16.0, Q=8.0, nsteps=30000, rho_s=rho_s,
                   ux=np.zeros((1, nx)), uy=np.zeros((1, nx)), T=T)


def kh_shear_layer(n: int = 4096, seed: int = SEED, ny: int | None = None) -> Problem:
    """Kelvin-Helmholtz shear layer with the paper's geometry (section
    "Kelvin-Helmholtz instability"): two species, u_y = 0.5 tanh((x-x0)/w)
    with w = 8 dx, species mass fraction following the same tanh, interface
    x0(y) = nx/2 + A sin(2 pi y / ny) with A = 4 dx and a seeded phase;
    uniform p = 1 and T = 1; outflow in x, periodic in y; dx = 1e-3,
    dt = 1e-5, tau = 2e-5."""
    rng = np.random.default_rng(seed)
    nx = n
    ny = n if ny is None else ny
    ph = float(rng.uniform(0, 2 * math.pi))
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    x0 = nx / 2 + 4.0 * np.sin(2 * math.pi * y / ny + ph)
    t = np.tanh((x - x0) / 8.0)
    uy = 0.5 * t
    y1 = 0.5 * (1.0 + t)
    rho = np.ones((ny, nx))
    rho_s = np.stack([rho * (1.0 - y1), rho * y1])
    sp = [species(m=1.0, tau=2e-5), species(m=1.0, tau=2e-5)]
    return Problem(name=f"kh_{nx}x{ny}_s2", nx=nx, ny=ny, species=sp, dx=1e-3, dy=1e-3, dt=1e-5,
                   bc_x=OUTFLOW, bc_y=PERIODIC, nsteps=1000, rho_s=rho_s,
                   ux=np.zeros((ny, nx)), uy=uy, T=np.ones((ny, nx)))


def uniform(nx: int, ny: int, sp: List[SpeciesSpec], rho_s, ux=0.0, uy=0.0, T=1.0, **kw) -> Problem:
    rho_s = np.asarray(rho_s, dtype=np.float64)[:, None, None] * np.ones((1, ny, nx))
    return Problem(name=f"uniform_{nx}x{ny}", nx=nx, ny=ny, species=sp, rho_s=rho_s,
                   ux=np.full((ny, nx), float(ux)), uy=np.full((ny, nx), float(uy)),
                   T=np.full((ny, nx), float(T)), **kw)


def shock_instance(L: int, seed: int) -> Problem:
    """An L x L two-species Sod-type tube along x (the shock-tube states:
    rho = 1, p = 1 left of x = L/2, rho = 0.125, p = 0.1 right), with a
    small seeded transverse perturbation of the interface so that the
    instance is genuinely 2-D; outflow in x, periodic in y."""
    rng = np.random.default_rng(seed)
    ph = float(rng.uniform(0, 2 * math.pi))
    x = np.arange(L)[None, :] * np.ones((L, 1))
    y = np.arange(L)[:, None] * np.ones((1, L))
    x0 = L / 2 + 2.0 * np.sin(2 * math.pi * y / L + ph)
    left = x < x0
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    sp = [species(tau=2e-5), species(tau=2e-5)]
    return Problem(name=f"shock_{L}", nx=L, ny=L, species=sp, dx=1e-3, dy=1e-3, dt=1e-5, bc_x=OUTFLOW,
                   bc_y=PERIODIC, rho_s=np.stack([0.5 * rho, 0.5 * rho]), ux=np.zeros((L, L)),
                   uy=np.zeros((L, L)), T=p / rho)


def reactive_instance(L: int, seed: int) -> Problem:
    """An L x L two-species reactive gas, F -> P (a = -1, +1, m = 1 each,
    rate k n_F n_F exp(-E_a/T): fuel and oxidiser index the same species),
    premixed fuel at T = 1 with a hot product spot at the centre; seeded
    k_ov, E_a/R, Q; periodic in x and y."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    r2 = ((xx - L / 2) ** 2 + (yy - L / 2) ** 2) / (L / 8) ** 2
    hot = np.exp(-r2)
    yF = 0.95 - 0.9 * hot
    rho = np.ones((L, L))
    T = 1.0 + 0.8 * hot
    sp = [species(tau=2e-5, a=-1.0), species(tau=2e-5, a=1.0)]
    return Problem(name=f"reactive_{L}", nx=L, ny=L, species=sp, dx=1e-3, dy=1e-3, dt=1e-5, bc_x=PERIODIC,
                   bc_y=PERIODIC, fuel=0, oxid=0, k_ov=float(rng.uniform(20.0, 40.0)),
                   Ea_over_R=float(rng.uniform(2.0, 3.0)), Q=float(rng.uniform(0.3, 0.6)),
                   rho_s=np.stack([rho * yF, rho * (1.0 - yF)]), ux=np.zeros((L, L)), uy=np.zeros((L, L)), T=T)


def batched_instances(n: int = 64, seed: int = SEED, lo: int = 64, hi: int = 512):
    """The batched workload: n independent two-species instances, sides
    drawn uniformly in [lo, hi] from the seed, alternately shock tubes and
    reactive gases; each also gets a seeded step count in [1000, 2000]."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        L = int(rng.integers(lo, hi + 1))
        pb = shock_instance(L, seed + k) if k % 2 == 0 else reactive_instance(L, seed + k)
        pb.nsteps = int(rng.integers(1000, 2001))
        out.append(pb)
    return out


# ---------------------------------------------------------------------------
# serving: requests arriving over time
# ---------------------------------------------------------------------------

@dataclass
class RequestSpec:
    """One serving request: an L x L instance of ``ns`` species, a shock
    tube or a reactive gas, advanced by ``nsteps`` steps; ``arrival`` in
    seconds after the start of the run; ``cancel_at`` (seconds after the
    start, or None) withdraws the request at that time."""
    rid: int
    kind: str
    L: int
    ns: int
    seed: int
    nsteps: int
    arrival: float = 0.0
    cancel_at: Optional[float] = None

    @property
    def units(self) -> int:  # species-cell updates the request asks for
        return self.L * self.L * self.ns * self.nsteps

    @property
    def cells(self) -> int:
        return self.L * self.L


def serving_requests(n: int = 200, seed: int = SEED, lo: int = 128, hi: int = 2048, steps=(1000, 10000),
                     species_counts=(2, 3, 4), reactive_frac: float = 0.5) -> List[RequestSpec]:
    """The serving mix: sides log-uniform in [lo, hi], species count uniform
    over ``species_counts``, a fraction ``reactive_frac`` reactive gases (the
    rest shock tubes), step counts uniform in ``steps`` (inclusive).
    Arrival times are left at 0 (the caller draws them)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        L = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        ns = int(rng.choice(species_counts))
        kind = "reactive" if rng.uniform() < reactive_frac else "shock"
        nsteps = int(rng.integers(steps[0], steps[1] + 1))
        out.append(RequestSpec(rid=k, kind=kind, L=L, ns=ns, seed=int(rng.integers(0, 2**31)), nsteps=nsteps))
    return out


def poisson_arrivals(specs: List[RequestSpec], rate: float, seed: int = SEED) -> List[RequestSpec]:
    """Copies of ``specs`` with Poisson arrivals at ``rate`` per second
    (exponential gaps, the first request at its gap after t = 0)."""
    rng = np.random.default_rng(seed + 1)
    t = 0.0
    out = []
    for s in specs:
        t += float(rng.exponential(1.0 / rate)) if rate > 0 else 0.0
        out.append(replace(s, arrival=t))
    return out


def _stoich(ns: int):
    """Fuel, oxidiser and stoichiometric coefficients of the one-step
    reaction of an ns-species request (equal masses, so sum a m = 0)."""
    if ns == 1:
        return 0, 0, [0.0]
    if ns == 2:
        return 0, 0, [-1.0, 1.0]  # F -> P, rate k n_F n_F exp(-E_a/T)
    if ns == 3:
        return 0, 1, [-1.0, -1.0, 2.0]
    a = [-1.0, -1.0] + [2.0 / (ns - 2)] * (ns - 2)
    return 0, 1, a


def request_problem(spec: RequestSpec) -> Problem:
    """The problem of a request without its initial fields (those come from
    ``request_fields``, on any device)."""
    rng = np.random.default_rng(spec.seed)
    L, ns = spec.L, spec.ns
    if spec.kind == "reactive":
        fuel, oxid, a = _stoich(ns)
        sp = [species(tau=2e-5, a=a[s]) for s in range(ns)]
        return Problem(name=f"req{spec.rid}_reactive_{L}_s{ns}", nx=L, ny=L, species=sp, dx=1e-3, dy=1e-3,
                       dt=1e-5, bc_x=PERIODIC, bc_y=PERIODIC, fuel=fuel, oxid=oxid,
                       k_ov=float(rng.uniform(20.0, 40.0)), Ea_over_R=float(rng.uniform(2.0, 3.0)),
                       Q=float(rng.uniform(0.3, 0.6)), nsteps=spec.nsteps)
    sp = [species(tau=2e-5) for _ in range(ns)]
    return Problem(name=f"req{spec.rid}_shock_{L}_s{ns}", nx=L, ny=L, species=sp, dx=1e-3, dy=1e-3, dt=1e-5,
                   bc_x=OUTFLOW, bc_y=PERIODIC, nsteps=spec.nsteps)


def request_fields(spec: RequestSpec, device="cpu"):
    """Initial fields (rho_s (S, L, L), ux, uy, T) of a request as FP64 torch
    tensors on ``device``: a Sod-type tube along x with a seeded transverse
    perturbation of the interface (shock), or a premixed gas with a hot
    product spot at the centre (reactive)."""
    import torch

    rng = np.random.default_rng(spec.seed + 7)
    L, ns = spec.L, spec.ns
    f64 = dict(dtype=torch.float64, device=device)
    y = torch.arange(L, **f64)[:, None].expand(L, L)
    x = torch.arange(L, **f64)[None, :].expand(L, L)
    zero = torch.zeros((L, L), **f64)
    if spec.kind == "reactive":
        fuel, oxid, a = _stoich(ns)
        r2 = ((x - L / 2) ** 2 + (y - L / 2) ** 2) / (L / 8) ** 2
        hot = torch.exp(-r2)
        reac = 0.95 - 0.9 * hot  # reactant mass fraction
        reactants = [s for s in range(ns) if a[s] < 0]
        products = [s for s in range(ns) if a[s] > 0]
        rho_s = torch.empty((ns, L, L), **f64)
        for s in range(ns):
            if s in reactants:
                rho_s[s] = reac / len(reactants)
            else:
                rho_s[s] = (1.0 - reac) / len(products)
        return rho_s, zero, zero.clone(), 1.0 + 0.8 * hot
    ph = float(rng.uniform(0, 2 * math.pi))
    x0 = L / 2 + 2.0 * torch.sin(2 * math.pi * y / L + ph)
    left = x < x0
    rho = torch.where(left, 1.0, 0.125).to(**f64)
    p = torch.where(left, 1.0, 0.1).to(**f64)
    rho_s = (rho / ns).unsqueeze(0).repeat(ns, 1, 1)
    return rho_s, zero, zero.clone(), p / rho


def air_shock(nx: int = 600, nsteps: int = 12000) -> Problem:
    """The air shock of section "Shock wave" (Eq. ConfigurationShock):
    79 % N2 / 21 % O2 by mole (diatomic, I = 3), pre-shock air at rest
    (1.17092 kg/m^3, 300 K) to the right of x0 = nx/4, the printed post-shock
    state (1.58407 kg/m^3, 106.637 m/s, 333.612 K) to the left.  Units: the
    pre-shock density and temperature, the molar mass of air (0.02885 kg/mol,
    so that the mean particle mass is 1) and the speed sqrt(R T / M_air) =
    294.04 m/s; then m_N2 = 0.97100, m_O2 = 1.10914.  Outflow in x, one row."""
    Rg, M_air = 8.314462618, 0.02885
    c_ref = math.sqrt(Rg * 300.0 / M_air)
    mN2, mO2 = 0.0280134 / M_air, 0.0319988 / M_air
    yN2 = 0.79 * mN2  # mass fractions (mean particle mass 1)
    yO2 = 0.21 * mO2
    rho_l, u_l, T_l = 1.58407 / 1.17092, 106.637 / c_ref, 333.612 / 300.0
    x = np.arange(nx)[None, :]
    left = x < nx // 4
    rho = np.where(left, rho_l, 1.0)
    ux = np.where(left, u_l, 0.0)
    T = np.where(left, T_l, 1.0)
    sp = [species(m=mN2, I=3.0, tau=2e-5), species(m=mO2, I=3.0, tau=2e-5)]
    return Problem(name=f"air_shock_{nx}", nx=nx, ny=1, species=sp, dx=1e-3, dy=1e-3, dt=1e-5, bc_x=OUTFLOW,
                   bc_y=PERIODIC, nsteps=nsteps, rho_s=np.stack([yN2 * rho, yO2 * rho]).astype(np.float64),
                   ux=ux.astype(np.float64), uy=np.zeros((1, nx)), T=T.astype(np.float64))
