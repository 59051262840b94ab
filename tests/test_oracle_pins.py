"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's own formulas: each checks the oracle
against an independent fact (a quadrature of the continuous Maxwellian, a
library inverse, a conservation law, a textbook scheme it must reduce to,
an exact Riemann solution, a Chapman-Enskog transport coefficient, a
closed-form special case, or a value printed in the paper).
"""
import math
import os

import numpy as np
import pytest

from paper_2006_15932_gb300 import workloads as W
from tests import riemann_exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sp(O, **kw):
    return O.Species(**kw)


def _species_list(O, n=3):
    # unequal masses, internal degrees of freedom, relaxation times and rings
    return [
        O.Species(m=1.0, I=3.0, tau=2e-5, v=(1.3, 1.2, 2.9, 2.4), eta=(2.2, 0.7, 0.4, 0.3)),
        O.Species(m=2.0, I=2.0, tau=3e-5, v=(0.9, 0.8, 2.1, 1.7), eta=(1.5, 0.5, 0.3, 0.2)),
        O.Species(m=0.5, I=4.0, tau=1.5e-5, v=(1.8, 1.7, 4.1, 3.4), eta=(3.3, 1.0, 0.6, 0.4)),
    ][:n]


# ---------------------------------------------------------------------------
# Equilibrium: the discrete moments equal those of the continuous Maxwellian
# (Eq. FormulaFeq and Eqs. relation1..relation7)
# ---------------------------------------------------------------------------

def _maxwellian_moment(phi, n, ux, uy, T, m, I, order=10):
    """Integral of phi(vx, vy, eta) f^eq over vx, vy, eta for the Maxwellian
    of Eq. FormulaFeq, by tensor Gauss-Hermite quadrature (exact for the
    polynomial moments used here)."""
    z, w = np.polynomial.hermite.hermgauss(order)
    sv = math.sqrt(2.0 * T / m)
    se = math.sqrt(2.0 * I * T / m)
    tot = 0.0
    for a, wa in zip(z, w):
        for b, wb in zip(z, w):
            for c, wc in zip(z, w):
                tot += wa * wb * wc * phi(ux + sv * a, uy + sv * b, se * c)
    return n * tot / math.pi ** 1.5


def _tensor_moments(vx, vy, eta, weights):
    """The 7 moment relations' left-hand sides, in tensor form: 1, v, v.v+eta^2,
    vv, (v.v+eta^2)v, vvv, (v.v+eta^2)vv, flattened over all components."""
    v = np.stack([vx, vy], axis=1)  # (Q, 2)
    q = vx ** 2 + vy ** 2 + eta ** 2
    out = [np.sum(weights)]
    out += list(np.einsum("i,ia->a", weights, v))
    out += [np.sum(weights * q)]
    out += list(np.einsum("i,ia,ib->ab", weights, v, v).ravel())
    out += list(np.einsum("i,i,ia->a", weights, q, v))
    out += list(np.einsum("i,ia,ib,ic->abc", weights, v, v, v).ravel())
    out += list(np.einsum("i,i,ia,ib->ab", weights, q, v, v).ravel())
    return np.array(out)


def _maxwellian_tensor_moments(n, ux, uy, T, m, I):
    def mono(k):
        # enumerate the same components as _tensor_moments
        comps = []
        comps.append(lambda x, y, e: 1.0)
        comps.append(lambda x, y, e: x)
        comps.append(lambda x, y, e: y)
        comps.append(lambda x, y, e: x * x + y * y + e * e)
        for a in range(2):
            for b in range(2):
                comps.append(lambda x, y, e, a=a, b=b: (x, y)[a] * (x, y)[b])
        for a in range(2):
            comps.append(lambda x, y, e, a=a: (x * x + y * y + e * e) * (x, y)[a])
        for a in range(2):
            for b in range(2):
                for c in range(2):
                    comps.append(lambda x, y, e, a=a, b=b, c=c: (x, y)[a] * (x, y)[b] * (x, y)[c])
        for a in range(2):
            for b in range(2):
                comps.append(lambda x, y, e, a=a, b=b: (x * x + y * y + e * e) * (x, y)[a] * (x, y)[b])
        return comps

    return np.array([_maxwellian_moment(phi, n, ux, uy, T, m, I) for phi in mono(None)])


@pytest.mark.parametrize("state", [(1.0, 0.0, 0.0, 1.0), (1.3, 0.21, -0.13, 0.87), (0.4, -0.5, 0.35, 1.6)])
@pytest.mark.parametrize("k", [0, 1, 2])
def test_feq_reproduces_maxwellian_moments(orc, state, k):
    sp = _species_list(orc)[k]
    n, ux, uy, T = state
    feq = orc.feq(sp, n, ux, uy, T)
    vx, vy, eta = orc.velocities(sp)
    got = _tensor_moments(vx, vy, eta, feq)
    want = _maxwellian_tensor_moments(n, ux, uy, T, sp.m, sp.I)
    scale = np.maximum(np.abs(want), 1.0)
    assert np.max(np.abs(got - want) / scale) < 1e-12


def test_velocity_set_structure(orc):
    """D2V16: four rings of four, two along the axes and two along the
    diagonals, each ring closed under 90-degree rotation."""
    sp = _species_list(orc)[0]
    vx, vy, eta = orc.velocities(sp)
    for r in range(4):
        ring = list(zip(vx[4 * r:4 * r + 4], vy[4 * r:4 * r + 4]))
        speed = sp.v[r] * (1.0 if r % 2 == 0 else math.sqrt(2.0))
        assert np.allclose([math.hypot(*p) for p in ring], speed, rtol=0, atol=1e-15)
        rot = {(round(-y, 12), round(x, 12)) for x, y in ring}
        assert rot == {(round(x, 12), round(y, 12)) for x, y in ring}
        assert np.all(eta[4 * r:4 * r + 4] == sp.eta[r])


def test_inverse_matches_library(orc):
    for sp in _species_list(orc):
        M = orc.moment_matrix(sp)
        Mi = orc.invert(M)
        ref = np.linalg.inv(M)
        assert np.max(np.abs(Mi - ref)) / np.max(np.abs(ref)) < 1e-12
        assert np.max(np.abs(M @ Mi - np.eye(16))) < 1e-11


def _exact_inverse(M):
    """Gauss-Jordan on exact rationals (every double is a rational), then
    each entry rounded to the nearest double by float(Fraction)."""
    from fractions import Fraction

    n = M.shape[0]
    A = [[Fraction(float(M[r, c])) for c in range(n)] + [Fraction(int(r == c)) for c in range(n)]
         for r in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if A[r][col] != 0)
        A[col], A[piv] = A[piv], A[col]
        p = A[col][col]
        A[col] = [x / p for x in A[col]]
        for r in range(n):
            if r != col and A[r][col] != 0:
                fac = A[r][col]
                A[r] = [a - fac * b for a, b in zip(A[r], A[col])]
    return np.array([[float(A[r][n + c]) for c in range(n)] for r in range(n)])


def test_minv_is_the_correctly_rounded_exact_inverse(orc):
    """f^eq = M^-1 f-hat with M^-1 rounded correctly from the exact inverse
    of M: every nonzero entry equals the exact rational inverse rounded to
    double; the structural zeros of the D2V16 symmetry stay below 1e-30 of
    the largest entry."""
    for sp in _species_list(orc, 3):
        E = _exact_inverse(orc.moment_matrix(sp))
        Mi = orc.minv(orc.Params(nx=1, ny=1, species=[sp]))[0]
        nz = E != 0
        assert np.array_equal(Mi[nz], E[nz])
        assert np.max(np.abs(Mi[~nz])) <= 1e-30 * np.max(np.abs(E))
        assert nz.sum() == 208


def test_all_eta_zero_is_singular(orc):
    sp = orc.Species(eta=(0.0, 0.0, 0.0, 0.0))
    M = orc.moment_matrix(sp)
    assert np.linalg.matrix_rank(M) < 16


def test_paper_duplicate_row_would_be_singular(orc):
    """The M_9 row printed as a copy of M_8 makes M singular; the oracle's
    reading (v.v + eta^2) v_y gives a full-rank matrix."""
    sp = _species_list(orc)[0]
    M = orc.moment_matrix(sp)
    assert np.linalg.matrix_rank(M) == 16
    bad = M.copy()
    bad[8] = bad[7]
    assert np.linalg.matrix_rank(bad) < 16


# ---------------------------------------------------------------------------
# Collision, reaction and force terms (Eqs. CollisionTerm, ReactionTerm,
# ForceTerm)
# ---------------------------------------------------------------------------

def _random_cell(O, sps, rng, rel=0.2):
    f = []
    for sp in sps:
        n = rng.uniform(0.3, 1.2)
        u = rng.uniform(-0.3, 0.3, size=2)
        T = rng.uniform(0.7, 1.3)
        fe = O.feq(sp, n, u[0], u[1], T)
        f.append(fe + rel * n / 16 * rng.uniform(-1, 1, size=16))
    return np.array(f)


def _sums(O, p, f, rhs):
    mass, mom, en = [], np.zeros(2), 0.0
    scale_m, scale_e = 0.0, 0.0
    for s, sp in enumerate(p.species):
        vx, vy, eta = O.velocities(sp)
        q = vx ** 2 + vy ** 2 + eta ** 2
        mass.append(np.sum(rhs[s]))
        mom += sp.m * np.array([np.sum(rhs[s] * vx), np.sum(rhs[s] * vy)])
        en += 0.5 * sp.m * np.sum(rhs[s] * q)
        scale_m += sp.m * np.sum(np.abs(rhs[s]) * (np.abs(vx) + np.abs(vy)))
        scale_e += 0.5 * sp.m * np.sum(np.abs(rhs[s]) * q)
    return np.array(mass), mom, en, scale_m, scale_e


def test_collision_conserves_mass_momentum_energy(orc):
    rng = np.random.default_rng(1)
    for trial in range(20):
        sps = _species_list(orc, 3)
        p = orc.Params(nx=1, ny=1, species=sps)
        f = _random_cell(orc, sps, rng)
        rhs, st = orc.cell_rhs(p, f)
        assert st == 0
        mass, mom, en, sm, se = _sums(orc, p, f, rhs)
        smass = np.sum(np.abs(rhs), axis=1)
        assert np.all(np.abs(mass) <= 1e-13 * smass)
        assert np.all(np.abs(mom) <= 1e-13 * sm)
        assert abs(en) <= 1e-13 * se


def test_collision_vanishes_at_equilibrium(orc):
    sps = _species_list(orc, 3)
    p = orc.Params(nx=1, ny=1, species=sps)
    f = np.array([orc.feq(sp, 0.4 + 0.2 * k, 0.12, -0.07, 1.1) for k, sp in enumerate(sps)])
    rhs, st = orc.cell_rhs(p, f)
    assert st == 0
    assert np.max(np.abs(rhs)) * sps[0].tau < 1e-14 * np.max(np.abs(f))


def _reactive_params(O, Q=1.5, k_ov=2e3, Ea=2.0):
    sps = [O.Species(m=1.0, I=3.0, tau=2e-5, a=-1.0),
           O.Species(m=2.0, I=2.0, tau=2e-5, a=-2.0, v=(0.9, 0.8, 2.1, 1.7), eta=(1.5, 0.5, 0.3, 0.2)),
           O.Species(m=5.0 / 3.0, I=4.0, tau=2e-5, a=3.0, v=(1.0, 0.9, 2.2, 1.9), eta=(1.7, 0.5, 0.3, 0.2))]
    # sum a m = -1 - 4 + 5 = 0
    return O.Params(nx=1, ny=1, species=sps, fuel=0, oxid=1, k_ov=k_ov, Ea_over_R=Ea, Q=Q)


def test_arrhenius_rate_special_cases(orc):
    p = _reactive_params(orc, Ea=0.0, k_ov=7.0)
    n = np.array([0.3, 0.5, 0.2])
    assert orc.omega(p, n, 1.0) == pytest.approx(7.0 * 0.3 * 0.5, rel=1e-15)
    assert orc.omega(p, n, 3.0) == pytest.approx(7.0 * 0.3 * 0.5, rel=1e-15)
    p = _reactive_params(orc, Ea=2.0, k_ov=7.0)
    r = orc.omega(p, n, 1.0) / orc.omega(p, n, 2.0)
    assert r == pytest.approx(math.exp(-2.0 * (1.0 - 0.5)), rel=1e-14)
    assert orc.omega(p, 2 * n, 1.0) == pytest.approx(4 * orc.omega(p, n, 1.0), rel=1e-15)
    p0 = _reactive_params(orc, k_ov=0.0)
    assert orc.omega(p0, n, 1.0) == 0.0


def test_reaction_term_mass_and_momentum(orc):
    """At equilibrium Omega = G = 0 and the rhs is R alone: sum_i R^s_i =
    a^s omega_ov (molar rate of species s) and the reaction moves no net
    mass or momentum because sum_s a^s m^s = 0."""
    p = _reactive_params(orc)
    n = [0.35, 0.5, 0.25]
    u, T = (0.1, -0.2), 1.2
    f = np.array([orc.feq(sp, n[s], u[0], u[1], T) for s, sp in enumerate(p.species)])
    rhs, st = orc.cell_rhs(p, f)
    assert st == 0
    w = orc.omega(p, np.array(n), T)
    assert w > 0
    for s, sp in enumerate(p.species):
        assert np.sum(rhs[s]) == pytest.approx(sp.a * w, rel=1e-11)
    mass, mom, en, sm, se = _sums(orc, p, f, rhs)
    assert abs(sum(sp.m * mass[s] for s, sp in enumerate(p.species))) < 1e-12 * w
    # momentum of the reaction: sum_s m^s a^s omega u = 0
    assert np.max(np.abs(mom)) < 1e-11 * sm


def test_reaction_energy_exact_when_temperature_is_steady(orc):
    """When the heat release exactly pays for the heat capacity change
    (Q = (T/2) sum_s (D+I^s) a^s, so T' = 0), the reaction term's energy
    rate is exactly Q omega_ov."""
    p = _reactive_params(orc)
    n = np.array([0.35, 0.5, 0.25])
    T = 1.2
    Qs = 0.5 * T * sum((2.0 + sp.I) * sp.a for sp in p.species)
    p.Q = Qs
    f = np.array([orc.feq(sp, n[s], 0.0, 0.0, T) for s, sp in enumerate(p.species)])
    rhs, st = orc.cell_rhs(p, f)
    w = orc.omega(p, n, T)
    assert orc.dTdt(p, n, T, w) == pytest.approx(0.0, abs=1e-12)
    _, _, en, _, se = _sums(orc, p, f, rhs)
    assert en == pytest.approx(Qs * w, rel=1e-10)


def test_reaction_energy_tends_to_heat_release(orc):
    """For small tau the energy rate of the reaction term tends to Q omega_ov
    (the chemical heat), with a defect that is first order in tau."""
    defects = []
    for tau in (2e-4, 1e-4, 5e-5):
        p = _reactive_params(orc, Q=6.0)
        for sp in p.species:
            sp.tau = tau
        n = np.array([0.35, 0.5, 0.25])
        T = 1.2
        f = np.array([orc.feq(sp, n[s], 0.0, 0.0, T) for s, sp in enumerate(p.species)])
        rhs, _ = orc.cell_rhs(p, f)
        w = orc.omega(p, n, T)
        _, _, en, _, _ = _sums(orc, p, f, rhs)
        defects.append(abs(en - 6.0 * w) / (6.0 * w))
    assert defects[0] < 0.05
    assert defects[1] / defects[2] == pytest.approx(2.0, rel=1e-3)
    assert defects[0] / defects[1] == pytest.approx(2.0, rel=1e-3)


def test_force_term_momentum_source(orc):
    """sum_i G^s_i = 0 and sum_i m^s v_i G^s_i = rho^s a for every species,
    away from equilibrium too."""
    rng = np.random.default_rng(5)
    sps = _species_list(orc, 3)
    a = (3.0, -7.0)
    p = orc.Params(nx=1, ny=1, species=sps, accel=a)
    p0 = orc.Params(nx=1, ny=1, species=sps)
    f = _random_cell(orc, sps, rng)
    rhs, _ = orc.cell_rhs(p, f)
    rhs0, _ = orc.cell_rhs(p0, f)
    G = rhs - rhs0
    for s, sp in enumerate(sps):
        vx, vy, eta = orc.velocities(sp)
        n = np.sum(f[s])
        assert abs(np.sum(G[s])) < 1e-9 * np.sum(np.abs(G[s]))
        assert sp.m * np.sum(G[s] * vx) == pytest.approx(sp.m * n * a[0], rel=1e-9)
        assert sp.m * np.sum(G[s] * vy) == pytest.approx(sp.m * n * a[1], rel=1e-9)


# ---------------------------------------------------------------------------
# NND scheme (section "Numerical simulation")
# ---------------------------------------------------------------------------

def _muscl_minmod_dflux(c, w, h):
    """Textbook upwind MUSCL flux with the minmod slope limiter, which the NND
    flux reduces to for a constant advection speed c."""
    def mm(a, b):
        return np.where(a * b > 0, np.sign(a) * np.minimum(abs(a), abs(b)), 0.0)

    w = np.asarray(w, dtype=float)
    if c > 0:
        face = lambda j: c * (w[j] + 0.5 * mm(w[j] - w[j - 1], w[j + 1] - w[j]))
        return (face(2) - face(1)) / h
    if c < 0:
        face = lambda j: c * (w[j + 1] - 0.5 * mm(w[j + 1] - w[j], w[j + 2] - w[j + 1]))
        return (face(2) - face(1)) / h
    return 0.0


def test_minmod(orc):
    assert orc.minmod(1.0, 2.0) == 1.0
    assert orc.minmod(-3.0, -2.0) == -2.0
    assert orc.minmod(1.0, -2.0) == 0.0
    assert orc.minmod(0.0, 5.0) == 0.0


def test_nnd_reduces_to_muscl_minmod(orc):
    rng = np.random.default_rng(7)
    for _ in range(500):
        w = rng.normal(size=5)
        if rng.random() < 0.2:
            w = np.cumsum(np.abs(w))  # monotone data
        c = rng.choice([-1, 1]) * rng.uniform(0.1, 3.0)
        h = rng.uniform(0.1, 2.0)
        assert orc.nnd_dflux(c, w, h) == pytest.approx(_muscl_minmod_dflux(c, w, h), rel=1e-12, abs=1e-12)
    assert orc.nnd_dflux(0.0, rng.normal(size=5), 1.0) == 0.0


def test_nnd_exact_for_linear_data(orc):
    """On linear data the limiter is inactive and the derivative exact."""
    for c in (2.0, -1.5):
        w = 3.0 + 0.7 * np.arange(-2, 3) * 0.1
        assert orc.nnd_dflux(c, w, 0.1) == pytest.approx(c * 0.7, rel=1e-12)


def test_nnd_second_order_on_smooth_data(orc):
    errs = []
    for n in (32, 64, 128):
        h = 1.0 / n
        x = np.arange(n) * h
        f = np.sin(2 * math.pi * x)
        d = np.array([orc.nnd_dflux(1.3, f[(np.arange(j - 2, j + 3)) % n], h) for j in range(n)])
        errs.append(np.mean(np.abs(d - 1.3 * 2 * math.pi * np.cos(2 * math.pi * x))))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0


def test_nnd_is_total_variation_diminishing(orc):
    n, c, h = 80, -1.0, 1.0 / 80
    dt = 0.4 * h / abs(c)
    f = np.where((np.arange(n) > 20) & (np.arange(n) < 45), 1.0, 0.0)
    tv0 = np.sum(np.abs(np.diff(np.r_[f, f[0]])))
    for _ in range(60):
        d = np.array([orc.nnd_dflux(c, f[(np.arange(j - 2, j + 3)) % n], h) for j in range(n)])
        f = f - dt * d
        tv = np.sum(np.abs(np.diff(np.r_[f, f[0]])))
        assert tv <= tv0 + 1e-12
        assert f.min() >= -1e-12 and f.max() <= 1.0 + 1e-12
        tv0 = tv


# ---------------------------------------------------------------------------
# Whole-step properties
# ---------------------------------------------------------------------------

def test_uniform_equilibrium_is_invariant(orc):
    sps = [W.species(m=1.0, tau=2e-5), W.species(m=2.0, I=2.0, tau=3e-5)]
    for bc in ((W.PERIODIC, W.PERIODIC), (W.OUTFLOW, W.PERIODIC), (W.OUTFLOW, W.OUTFLOW)):
        pb = W.uniform(9, 7, sps, rho_s=[0.4, 0.7], ux=0.13, uy=-0.08, T=0.95, bc_x=bc[0], bc_y=bc[1])
        p = orc.params_of(pb)
        f0 = orc.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)
        f, st = orc.run(p, f0, 20)
        assert st == 0
        assert np.max(np.abs(f - f0)) <= 1e-13 * np.max(np.abs(f0))


def test_mass_and_momentum_conserved_on_periodic_grid(orc):
    pb = W.random_smooth(12, 10, 3, seed=3, unequal=True)
    p = orc.params_of(pb)
    f0 = orc.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)
    c0 = orc.conservation(p, f0)
    f, st = orc.run(p, f0, 25)
    assert st == 0
    c1 = orc.conservation(p, f)
    assert np.max(np.abs(c1[:3] - c0[:3]) / np.abs(c0[:3])) < 1e-13
    # momentum and energy: exact up to round-off summed over cells
    assert np.max(np.abs(c1[3:6] - c0[3:6])) < 1e-12 * np.max(np.abs(c0[3:6]))


def test_free_fall_velocity_is_a_t(orc):
    """Uniform box under a constant acceleration: the mixture velocity grows
    exactly as u_y = a t (the free-falling box of section "Combustion in
    constant volume"; golden values in tests/golden/free_fall.txt)."""
    gold = dict(l.split("=") for l in open(os.path.join(GOLDEN, "free_fall.txt"))
                if "=" in l and not l.startswith("#"))
    g, t_end, uy_exact = float(gold["g"]), float(gold["t"]), float(gold["uy_exact"])
    paper_rel = float(gold["d2v16_rel_err"])
    assert g * t_end == pytest.approx(uy_exact, rel=1e-12)
    # nondimensional stand-in: the same a*t law at 100 steps
    sps = [W.species(m=1.0, tau=2e-5), W.species(m=2.0, I=2.0, tau=3e-5)]
    a = -9.8
    pb = W.uniform(3, 3, sps, rho_s=[0.4, 0.9], T=1.0, accel=(0.0, a))
    p = orc.params_of(pb)
    f0 = orc.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)
    f, st = orc.run(p, f0, 100)
    assert st == 0
    mom = orc.moments(p, f)
    uy = mom[4 * 2 + 2]
    want = a * 100 * pb.dt
    assert np.max(np.abs(uy - want)) <= 1e-9 * abs(want)
    # at least as accurate as the paper's D2V16 run
    assert np.max(np.abs(uy - want)) / abs(want) < paper_rel


def test_reactive_uniform_box_budget(orc):
    """Uniform reactive box: each species' moles change by dt a^s omega_ov per
    step, total mass is constant, and thermal energy plus the heat bound in
    the fuel changes only by the first-order-in-tau defect of the reaction
    term."""
    sps = [W.species(tau=2e-5, a=-1.0), W.species(tau=2e-5, a=-1.0), W.species(tau=2e-5, a=2.0)]
    pb = W.uniform(2, 2, sps, rho_s=[0.45, 0.45, 0.1], T=1.3, fuel=0, oxid=1, k_ov=50.0,
                   Ea_over_R=2.0, Q=0.8)
    p = orc.params_of(pb)
    f = orc.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)
    c0 = orc.conservation(p, f)
    for _ in range(5):
        m0 = orc.moments(p, f)
        n = m0[[0, 4, 8], 0, 0]
        T = m0[4 * 3 + 3, 0, 0]
        w = orc.omega(p, n, T)
        f, st = orc.run(p, f, 1)
        assert st == 0
        m1 = orc.moments(p, f)
        for s, sp in enumerate(sps):
            assert m1[4 * s, 0, 0] - n[s] == pytest.approx(pb.dt * sp.a * w, rel=1e-8)
    c1 = orc.conservation(p, f)
    assert sum(c1[:3]) == pytest.approx(sum(c0[:3]), rel=1e-14)
    e0, e1 = c0[3 + 2] + c0[3 + 3], c1[3 + 2] + c1[3 + 3]
    released = c0[3 + 3] - c1[3 + 3]
    assert released > 0
    assert abs(e1 - e0) < 0.01 * released


def test_status_flags_bad_input(orc):
    sps = [W.species(), W.species()]
    pb = W.uniform(4, 1, sps, rho_s=[0.5, 0.5], T=1.0)
    p = orc.params_of(pb)
    f = orc.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)
    f[0, :, 0, 2] = -f[0, :, 0, 2]
    _, st = orc.run(p, f, 1)
    assert st & 1


# ---------------------------------------------------------------------------
# Hydrodynamic limit
# ---------------------------------------------------------------------------

def test_riemann_helper_textbook_star_state():
    p, u = riemann_exact.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4)
    assert p == pytest.approx(0.30313, abs=1e-5)
    assert u == pytest.approx(0.92745, abs=1e-5)


def test_paper_shock_states_satisfy_rankine_hugoniot():
    """The pre/post-shock states printed for the air shock (section "Shock
    wave", tests/golden/shock_air.txt) conserve mass and momentum across a
    steady shock: this checks the golden fixture and the reading of its
    units (p = rho R T / M with the molar mass of air)."""
    gold = dict(l.split("=") for l in open(os.path.join(GOLDEN, "shock_air.txt"))
                if "=" in l and not l.startswith("#"))
    rl, ul, Tl = (float(gold[k]) for k in ("rho_L", "ux_L", "T_L"))
    rr, ur, Tr = (float(gold[k]) for k in ("rho_R", "ux_R", "T_R"))
    Rg, Mair, pr = 8.314462618, float(gold["M_air"]), 101325.0
    s = rl * ul / (rl - rr)  # shock speed from mass conservation
    pl = pr + rr * s * ul  # momentum conservation
    assert pl == pytest.approx(rl * Rg * Tl / Mair, rel=2e-3)
    assert pr == pytest.approx(rr * Rg * Tr / Mair, rel=2e-3)


@pytest.mark.slow
def test_sod_shock_tube_against_exact_riemann(orc):
    pb = W.sod_tube(400, 2000)
    p = orc.params_of(pb)
    f0 = orc.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)
    f, st = orc.run(p, f0, pb.nsteps)
    assert st == 0
    m = orc.moments(p, f)
    rho, ux, pr = m[8, 0], m[9, 0], m[12, 0]
    t = pb.nsteps * pb.dt
    x = (np.arange(pb.nx) + 0.5) * pb.dx
    er, eu, ep = riemann_exact.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 1.4, (x - 0.2) / t)
    l1 = lambda a, b: np.mean(np.abs(a - b))
    # measured on the oracle: 0.0024, 0.0045, 0.0019 (mostly NND smearing of
    # the contact and the shock over a few cells)
    assert l1(rho, er) < 0.004
    assert l1(ux, eu) < 0.007
    assert l1(pr, ep) < 0.003
    # far-field states untouched, mass conserved by the outflow faces
    assert abs(rho[5] - 1.0) < 1e-6 and abs(rho[-5] - 0.125) < 1e-6


@pytest.mark.slow
def test_shear_wave_viscosity(orc):
    """Decaying transverse shear wave u_y = U sin(k x) exp(-nu k^2 t): the
    measured nu matches the Chapman-Enskog value nu = mu/rho = tau T/m
    (mu = p tau, below Eq. NS3)."""
    nx = 256
    L = 1.0
    dx = L / nx
    tau, T, m = 0.004, 1.0, 1.0
    sp = [W.species(m=m, tau=tau)]
    x = (np.arange(nx) + 0.5) * dx
    U = 0.01
    k = 2 * math.pi / L
    dt = 0.2 * dx / 2.9
    pb = W.Problem(name="shear", nx=nx, ny=1, species=sp, dx=dx, dy=dx, dt=dt,
                   rho_s=np.ones((1, 1, nx)), ux=np.zeros((1, nx)),
                   uy=(U * np.sin(k * x))[None, :], T=np.full((1, nx), T))
    p = orc.params_of(pb)
    f = orc.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)
    amps, times = [], []
    nsteps = int(round(0.4 / (2 * math.pi) ** 2 / (tau * T / m) / dt))
    chunk = nsteps // 4
    for c in range(5):
        uy = orc.moments(p, f)[4 + 2, 0]
        amps.append(2.0 / nx * np.sum(uy * np.sin(k * x)))
        times.append(c * chunk * dt)
        if c < 4:
            f, st = orc.run(p, f, chunk)
            assert st == 0
    rate = -np.polyfit(times[1:], np.log(amps[1:]), 1)[0]
    nu = rate / k ** 2
    print("measured nu", nu, "Chapman-Enskog", tau * T / m)
    assert nu == pytest.approx(tau * T / m, rel=0.01)  # measured: 0.03 %


# ---------------------------------------------------------------------------
# Outputs: macroscopic fields and the nonequilibrium moments (Eqs. Delta2,
# Delta31, Delta3, Delta42 and the energy diagnostics that follow them)
# ---------------------------------------------------------------------------

def _equilibrium_state(orc, ns=3, nx=9, ny=7, seed=4):
    pb = W.random_smooth(nx, ny, ns, seed=seed)
    p = orc.params_of(pb)
    return pb, p, orc.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)


def _rel(a, b, scale):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / scale)


def test_moments_of_the_equilibrium_are_its_fields(orc):
    """f^eq built from (rho^s, u, T) has exactly those moments: n^s =
    rho^s / m^s, u^s = u and T^s = T for every species, and the mixture
    rho = sum rho^s, u, T and p = n T."""
    pb, p, f = _equilibrium_state(orc)
    mom = orc.moments(p, f)
    S = pb.ns
    m = np.array([sp.m for sp in pb.species])[:, None, None]
    n = pb.rho_s / m
    uscale = max(np.max(np.abs(pb.ux)), np.max(np.abs(pb.uy)))
    for s in range(S):
        assert _rel(mom[4 * s], n[s], np.max(n[s])) < 1e-12
        assert _rel(mom[4 * s + 1], pb.ux, uscale) < 1e-12
        assert _rel(mom[4 * s + 2], pb.uy, uscale) < 1e-12
        assert _rel(mom[4 * s + 3], pb.T, np.max(pb.T)) < 1e-12
    rho = pb.rho_s.sum(axis=0)
    assert _rel(mom[4 * S], rho, np.max(rho)) < 1e-12
    assert _rel(mom[4 * S + 1], pb.ux, uscale) < 1e-12
    assert _rel(mom[4 * S + 2], pb.uy, uscale) < 1e-12
    assert _rel(mom[4 * S + 3], pb.T, np.max(pb.T)) < 1e-12
    pr = n.sum(axis=0) * pb.T
    assert _rel(mom[4 * S + 4], pr, np.max(pr)) < 1e-12


def test_nonequilibrium_moments_vanish_at_equilibrium(orc):
    """For f = f^eq every Delta is zero, M(f) equals M(f^eq), and the
    equilibrium diagnostics take their closed forms (D = 2):
    M_2aa(f^eq)/2 = (n T + rho u_a^2)/2 and
    M_3,1a(f^eq)/2 = rho u_a ((D + I + 2) T/m + u.u)/2."""
    pb, p, f = _equilibrium_state(orc)
    d = orc.nonequilibrium(p, f)
    u2 = pb.ux ** 2 + pb.uy ** 2
    for s, sp in enumerate(pb.species):
        rows = d[20 * s:20 * s + 20]
        scale = np.max(np.abs(rows[12:20]))
        assert np.max(np.abs(rows[0:12])) / scale < 1e-12
        assert _rel(rows[12:14], rows[14:16], scale) < 1e-13
        assert _rel(rows[16:18], rows[18:20], scale) < 1e-13
        rho = pb.rho_s[s]
        n = rho / sp.m
        assert _rel(rows[14], 0.5 * (n * pb.T + rho * pb.ux ** 2), scale) < 1e-12
        assert _rel(rows[15], 0.5 * (n * pb.T + rho * pb.uy ** 2), scale) < 1e-12
        a2 = (2.0 + sp.I + 2.0) * pb.T / sp.m + u2
        assert _rel(rows[18], 0.5 * rho * pb.ux * a2, scale) < 1e-12
        assert _rel(rows[19], 0.5 * rho * pb.uy * a2, scale) < 1e-12


def _permutation(vx, vy, eta, image):
    """Index map i -> j of the velocity set with (vx_j, vy_j) = image(vx_i,
    vy_i) and the same internal speed."""
    perm = []
    for i in range(len(vx)):
        tx, ty = image(vx[i], vy[i])
        j = [k for k in range(len(vx))
             if abs(vx[k] - tx) < 1e-12 and abs(vy[k] - ty) < 1e-12 and eta[k] == eta[i]]
        assert len(j) == 1
        perm.append(j[0])
    return perm


def test_nonequilibrium_moments_follow_the_square_symmetries(orc):
    """Mirroring a nonequilibrium state in x (v_x -> -v_x) flips exactly the
    components odd in x; exchanging x and y exchanges the x and y
    components.  A wrong index or sign in any of the 20 sums fails one of
    the two."""
    pb, p, feq = _equilibrium_state(orc, ns=2, nx=5, ny=3, seed=8)
    rng = np.random.default_rng(9)
    f = feq * (1.0 + 0.1 * rng.uniform(-1, 1, size=feq.shape))
    d = orc.nonequilibrium(p, f)
    mirror_sign = np.array([1, -1, 1, -1, 1, -1, 1, -1, 1, 1, -1, 1, 1, 1, 1, 1, -1, 1, -1, 1])
    swap_rows = [2, 1, 0, 4, 3, 8, 7, 6, 5, 11, 10, 9, 13, 12, 15, 14, 17, 16, 19, 18]
    fm, fs = np.empty_like(f), np.empty_like(f)
    for s, sp in enumerate(pb.species):
        vx, vy, eta = orc.velocities(sp)
        pm = _permutation(vx, vy, eta, lambda x, y: (-x, y))
        ps = _permutation(vx, vy, eta, lambda x, y: (y, x))
        fm[s] = f[s][pm]
        fs[s] = f[s][ps]
    dm = orc.nonequilibrium(p, fm)
    ds = orc.nonequilibrium(p, fs)
    for s in range(pb.ns):
        rows = d[20 * s:20 * s + 20]
        scale = np.max(np.abs(rows))
        assert np.max(np.abs(rows[0:12])) / scale > 1e-4  # a real departure
        assert _rel(dm[20 * s:20 * s + 20], mirror_sign[:, None, None] * rows, scale) < 1e-12
        assert _rel(ds[20 * s:20 * s + 20], rows[swap_rows], scale) < 1e-12


def test_conserved_totals_of_the_equilibrium(orc):
    """The conserved totals of f^eq(rho^s, u, T) in closed form: species
    masses sum rho^s, momentum sum rho u, energy sum over species and cells
    of n^s (D + I^s) T / 2 + rho^s u.u / 2 (D = 2), and with a reaction the
    heat still bound in the fuel, Q n^fuel / |a^fuel| summed over cells."""
    pb = W.random_smooth(9, 7, 3, seed=5, reactive=True)
    p = orc.params_of(pb)
    f = orc.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)
    c = orc.conservation(p, f)
    S = pb.ns
    rho = pb.rho_s.sum(axis=0)
    u2 = pb.ux ** 2 + pb.uy ** 2
    want = [pb.rho_s[s].sum() for s in range(S)]
    want += [(rho * pb.ux).sum(), (rho * pb.uy).sum()]
    energy = sum(((pb.rho_s[s] / sp.m) * (2.0 + sp.I) * pb.T / 2 + pb.rho_s[s] * u2 / 2).sum()
                 for s, sp in enumerate(pb.species))
    fuel = pb.species[pb.fuel]
    bound = (pb.Q * (pb.rho_s[pb.fuel] / fuel.m) / abs(fuel.a)).sum()
    want += [energy, bound]
    want = np.array(want)
    scale = np.maximum(np.abs(want), np.max(np.abs(want[:S])))
    assert np.max(np.abs(c - want) / scale) < 1e-12, (c, want)


@pytest.mark.parametrize("bc", [(W.PERIODIC, W.PERIODIC), (W.OUTFLOW, W.PERIODIC), (W.PERIODIC, W.OUTFLOW)])
def test_step_region_is_a_window_of_the_full_step(orc, bc):
    """The windowed step (the reference of the sampled full-size GPU checks)
    equals the same window of one full-grid step, bit for bit, for windows
    touching every edge and one in the interior, with reaction and force."""
    pb = W.random_smooth(13, 11, 3, seed=7, reactive=True, force=True, bc=bc)
    p = orc.params_of(pb)
    rng = np.random.default_rng(2)
    f0 = orc.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)
    f0 = f0 * (1.0 + 0.05 * rng.uniform(-1, 1, size=f0.shape))
    full, st = orc.run(p, f0, 1)
    assert st == 0
    for (x0, x1, y0, y1) in [(0, 5, 0, 4), (8, 13, 7, 11), (0, 13, 5, 6), (4, 9, 3, 8), (12, 13, 0, 11)]:
        got, st = orc.step_region(p, f0, x0, x1, y0, y1)
        assert st == 0
        assert np.array_equal(got, full[:, :, y0:y1, x0:x1]), (x0, x1, y0, y1)
