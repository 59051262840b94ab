"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative L-inf = max|a - b| / max|b| per field):
  FP64: 1e-12 on f and on every output field.
  FP32: derived from float rounding: each step adds O(1e-7) relative
        rounding to f; with the relaxation and the advection contracting,
        the error grows at most linearly, so 50 steps stay below
        1e-7 * 50 * (a safety factor of 4) = 2e-5 on f and the
        conserved moments; the derived T and u have an extra factor of
        cond ~ 10 from the subtraction E/n - u^2 (bound 2e-4).
"""
import math

import numpy as np
import pytest

from paper_2006_15932_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL_F = 2e-5


def rel_linf(a, b, scale=None):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = max(np.max(np.abs(b)), 1e-300) if scale is None else scale
    return float(np.max(np.abs(a - b)) / den)


def moments_errors(mom, ref, ns):
    """Relative L-inf of every row of the moments output; velocity rows are
    measured against the flow's velocity scale (largest |u| component or
    the thermal speed sqrt(T/m)), so that a velocity component that is zero
    up to round-off is not divided by its own round-off."""
    T = ref[4 * ns + 3]
    vscale = max(np.max(np.abs(ref[4 * ns + 1])), np.max(np.abs(ref[4 * ns + 2])), np.sqrt(np.max(T)))
    errs = []
    for k in range(ref.shape[0]):
        is_vel = (k < 4 * ns and k % 4 in (1, 2)) or k in (4 * ns + 1, 4 * ns + 2)
        errs.append(rel_linf(mom[k], ref[k], vscale if is_vel else None))
    return np.array(errs)


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_15932_gb300 import build as B
    from paper_2006_15932_gb300 import dbm

    B.build()
    dbm.load()
    return dbm


def _oracle_f0(orc, pb):
    p = orc.params_of(pb)
    return p, orc.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)


def _noneq_f(orc, pb, seed=3, rel=0.05):
    """An oracle-built nonequilibrium state: f^eq of the problem's fields
    times (1 + rel * noise), so that every term of the step is active."""
    p, f0 = _oracle_f0(orc, pb)
    rng = np.random.default_rng(seed)
    return p, f0 * (1.0 + rel * rng.uniform(-1, 1, size=f0.shape))


# ---------------------------------------------------------------------------
# FP64: the configuration of the parity gate and random 2-D cases
# ---------------------------------------------------------------------------

def test_sod_tube_fp64_2000_steps(D, orc):
    pb = W.sod_tube(400, 2000)
    s = D.Solver(pb, "fp64")
    s.set_state()
    s.step(pb.nsteps)
    f = s.get_f().cpu().numpy()
    mom = s.moments().cpu().numpy()
    assert s.status()[0] == 0
    p, f0 = _oracle_f0(orc, pb)
    fr, st = orc.run(p, f0, pb.nsteps)
    assert st == 0
    mr = orc.moments(p, fr)
    assert rel_linf(f, fr) <= FP64_TOL
    errs = moments_errors(mom, mr, pb.ns)
    assert np.all(errs <= FP64_TOL), errs


@pytest.mark.parametrize("nx,ny,ns,bc,reactive,force", [
    (37, 11, 3, (W.OUTFLOW, W.PERIODIC), True, True),
    (33, 17, 2, (W.PERIODIC, W.PERIODIC), False, False),
    (64, 9, 1, (W.PERIODIC, W.OUTFLOW), False, True),
    (5, 40, 4, (W.OUTFLOW, W.OUTFLOW), True, False),
])
def test_random_fp64(D, orc, nx, ny, ns, bc, reactive, force):
    pb = W.random_smooth(nx, ny, ns, seed=nx * ny, reactive=reactive, force=force, bc=bc)
    p, f0 = _noneq_f(orc, pb)
    s = D.Solver(pb, "fp64")
    s.set_f(f0)
    s.step(30)
    f = s.get_f().cpu().numpy()
    fr, st = orc.run(p, f0, 30)
    assert st == 0 and s.status()[0] == 0
    assert rel_linf(f, fr) <= FP64_TOL


def test_set_state_matches_oracle_equilibrium(D, orc):
    pb = W.random_smooth(29, 13, 3, seed=5)
    s = D.Solver(pb, "fp64")
    s.set_state()
    p, f0 = _oracle_f0(orc, pb)
    assert rel_linf(s.get_f().cpu().numpy(), f0) <= FP64_TOL


def test_fp32_set_state_is_the_equilibrium(D, orc):
    """FP32 storage starts from the FP32 block solve of f^eq: a few float
    ulps from the oracle's FP64 equilibrium, and the conserved totals of the
    oracle's equilibrium to float rounding."""
    pb = W.random_smooth(41, 17, 3, seed=6, reactive=True)
    s = D.Solver(pb, "fp32")
    s.set_state()
    p, f0 = _oracle_f0(orc, pb)
    assert rel_linf(s.get_f().cpu().numpy(), f0) <= 1e-6
    c = s.conservation().cpu().numpy()
    cr = orc.conservation(p, f0)
    assert np.max(np.abs(c - cr) / np.maximum(np.abs(cr), 1e-30)) <= 1e-6


def test_outputs_fp64(D, orc):
    pb = W.random_smooth(31, 12, 3, seed=8, reactive=True)
    p, f0 = _noneq_f(orc, pb, rel=0.1)
    s = D.Solver(pb, "fp64")
    s.set_f(f0)
    mom = s.moments().cpu().numpy()
    neq = s.nonequilibrium().cpu().numpy()
    cons = s.conservation().cpu().numpy()
    mr = orc.moments(p, f0)
    nr = orc.nonequilibrium(p, f0)
    cr = orc.conservation(p, f0)
    errs = moments_errors(mom, mr, pb.ns)
    assert np.all(errs <= FP64_TOL), errs
    for k in range(nr.shape[0]):
        assert rel_linf(neq[k], nr[k]) <= 1e-11, ("noneq", k)
    assert np.max(np.abs(cons - cr) / np.maximum(np.abs(cr), 1e-300)) <= 1e-12


@pytest.mark.parametrize("nx,ny,bc", [(1, 1, (W.PERIODIC, W.PERIODIC)), (1, 3, (W.OUTFLOW, W.PERIODIC)),
                                      (2, 1, (W.PERIODIC, W.OUTFLOW)), (3, 2, (W.OUTFLOW, W.OUTFLOW))])
def test_degenerate_grids(D, orc, nx, ny, bc):
    pb = W.random_smooth(nx, ny, 2, seed=1, bc=bc)
    p, f0 = _noneq_f(orc, pb)
    s = D.Solver(pb, "fp64")
    s.set_f(f0)
    s.step(7)
    fr, st = orc.run(p, f0, 7)
    assert rel_linf(s.get_f().cpu().numpy(), fr) <= FP64_TOL


def test_eight_species(D, orc):
    pb = W.random_smooth(19, 6, 8, seed=2)
    p, f0 = _noneq_f(orc, pb)
    s = D.Solver(pb, "fp64")
    s.set_f(f0)
    s.step(5)
    fr, _ = orc.run(p, f0, 5)
    assert rel_linf(s.get_f().cpu().numpy(), fr) <= FP64_TOL


@pytest.mark.parametrize("ns,bc,force", [(5, (W.OUTFLOW, W.PERIODIC), True), (8, (W.PERIODIC, W.OUTFLOW), False)])
def test_fp32_many_species_against_oracle(D, orc, ns, bc, force):
    """Five and eight species in FP32 run the species-staged kernel (each
    species through shared memory on its own) by default: 20 steps against
    the oracle on a grid of two 64-wide tiles with ragged tails in x and y,
    force on for five species."""
    pb = W.random_smooth(70, 13, ns, seed=30 + ns, force=force, bc=bc)
    p, f0 = _noneq_f(orc, pb)
    s = D.Solver(pb, "fp32")
    assert s.step_tile() == (64, 8, 2)
    s.set_f(f0)
    s.step(20)
    f = s.get_f().cpu().numpy()
    mom = s.moments().cpu().numpy()
    assert s.status()[0] == 0
    fr, _ = orc.run(p, f0, 20)
    assert rel_linf(f, fr) <= FP32_TOL_F
    errs = moments_errors(mom, orc.moments(p, fr), pb.ns)
    assert np.all(errs <= 2e-4), errs


def test_staged_full_size_one_step_sampled(D, orc):
    """Six species on 1024 x 512 (1024 tiles of the species-staged kernel),
    one step, against the oracle on sampled windows (edges and interior)."""
    pb = W.random_smooth(1024, 512, 6, seed=36, bc=(W.OUTFLOW, W.PERIODIC))
    s = D.Solver(pb, "fp32")
    assert s.step_tile() == (64, 8, 2)
    s.set_state()
    f0 = s.get_f().cpu().numpy()
    s.step(1)
    f1 = s.get_f().cpu().numpy()
    assert s.status()[0] == 0
    s.close()
    p = orc.params_of(pb)
    rng = np.random.default_rng(1)
    for (x0, x1, y0, y1) in _windows(pb.nx, pb.ny, rng, k=3, w=20):
        want, st = orc.step_region(p, f0, x0, x1, y0, y1)
        assert st == 0
        assert rel_linf(f1[:, :, y0:y1, x0:x1], want) <= 1e-6, (x0, y0)


def test_zero_steps_is_identity(D, orc):
    pb = W.random_smooth(10, 4, 2, seed=4)
    p, f0 = _noneq_f(orc, pb)
    s = D.Solver(pb, "fp64")
    s.set_f(f0)
    s.step(0)
    assert np.array_equal(s.get_f().cpu().numpy(), f0)


def test_checkpoint_resume_is_bitwise(D, orc):
    pb = W.random_smooth(21, 9, 2, seed=6, reactive=False)
    for prec in ("fp64", "fp32"):
        a = D.Solver(pb, prec)
        a.set_state()
        a.step(10)
        a.step(10)
        fa = a.get_f().cpu().numpy()
        b = D.Solver(pb, prec)
        b.set_state()
        b.step(10)
        ck = b.get_f()
        c = D.Solver(pb, prec)
        c.set_f(ck)
        c.step(10)
        assert np.array_equal(c.get_f().cpu().numpy(), fa)


def test_health_flag_reports_negative_density(D, orc):
    pb = W.random_smooth(8, 8, 2, seed=9)
    p, f0 = _oracle_f0(orc, pb)
    f0[1, :, 3, 4] *= -1.0  # the host plants a negative density at one cell
    s = D.Solver(pb, "fp64")
    s.set_f(f0)
    s.step(1)
    rc, bits = s.status()
    assert rc == -6 and bits & 1
    s.set_state()  # a fresh state clears the flag
    s.step(1)
    assert s.status() == (0, 0)


# ---------------------------------------------------------------------------
# FP32
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("reactive", [False, True])
def test_fp32_against_oracle(D, orc, reactive):
    pb = W.random_smooth(70, 23, 3, seed=12, reactive=reactive, bc=(W.OUTFLOW, W.PERIODIC))
    p, f0 = _noneq_f(orc, pb)
    s = D.Solver(pb, "fp32")
    s.set_f(f0)
    s.step(50)
    f = s.get_f().cpu().numpy()
    mom = s.moments().cpu().numpy()
    fr, _ = orc.run(p, f0, 50)
    mr = orc.moments(p, fr)
    assert rel_linf(f, fr) <= FP32_TOL_F
    errs = moments_errors(mom, mr, pb.ns)
    assert np.all(errs <= 2e-4), errs


def test_fp32_conservation_drift(D, orc):
    pb = W.random_smooth(64, 64, 2, seed=13)
    s = D.Solver(pb, "fp32")
    s.set_state()
    c0 = s.conservation().cpu().numpy()
    s.step(200)
    c1 = s.conservation().cpu().numpy()
    assert np.max(np.abs(c1[:2] - c0[:2]) / np.abs(c0[:2])) < 1e-6
    assert abs(c1[4] - c0[4]) / abs(c0[4]) < 1e-6


def _two_species(nx, ny, bc, react, force, seed=23):
    """Two species on a smooth random state; with ``react`` the one-step
    reaction A + B -> 2 B (equal masses, so sum a m = 0), with ``force`` a
    body force: every branch of the two-species step."""
    pb = W.random_smooth(nx, ny, 2, seed=seed, force=force, bc=bc)
    if react:
        for sp in pb.species:
            sp.m = 1.0
        pb.species[0].a, pb.species[1].a = -1.0, 1.0
        pb.fuel, pb.oxid = 0, 1
        pb.k_ov, pb.Ea_over_R, pb.Q = 2.0e3, 2.0, 1.5
    return pb


@pytest.mark.parametrize("nx,ny,react", [(130, 21, True), (129, 9, False)])
def test_fp32_two_species_against_oracle(D, orc, nx, ny, react):
    """The two-species FP32 step (two cells per thread, packed FP32x2
    arithmetic) against the oracle: tiles of 64 x 4 cells with ragged tails
    in both directions, an odd nx (the last thread of a row has one cell),
    reaction and force on."""
    pb = _two_species(nx, ny, (W.OUTFLOW, W.PERIODIC), react, True)
    p, f0 = _noneq_f(orc, pb)
    s = D.Solver(pb, "fp32", step_kernel="tma_pair")
    assert s.step_tile() == (64, 8, 2)
    s.set_f(f0)
    s.step(50)
    f = s.get_f().cpu().numpy()
    mom = s.moments().cpu().numpy()
    assert s.status()[0] == 0
    fr, _ = orc.run(p, f0, 50)
    mr = orc.moments(p, fr)
    assert rel_linf(f, fr) <= FP32_TOL_F
    errs = moments_errors(mom, mr, pb.ns)
    assert np.all(errs <= 2e-4), errs


@pytest.mark.parametrize("nx,ny,bc,react,force", [(130, 11, (W.PERIODIC, W.PERIODIC), False, True),
                                                  (128, 9, (W.OUTFLOW, W.OUTFLOW), True, False),
                                                  (66, 7, (W.PERIODIC, W.OUTFLOW), True, True),
                                                  (129, 6, (W.OUTFLOW, W.PERIODIC), True, True),
                                                  (2, 2, (W.PERIODIC, W.PERIODIC), False, True),
                                                  (3, 5, (W.OUTFLOW, W.PERIODIC), True, False),
                                                  (1, 3, (W.PERIODIC, W.OUTFLOW), False, False),
                                                  (63, 4, (W.PERIODIC, W.PERIODIC), False, False)])
def test_pair_kernel_matches_generic(D, orc, nx, ny, bc, react, force):
    """The two-cells-per-thread kernel against the one-cell generic kernel
    after 6 steps, bit for bit (each half of a packed FP32x2 operation rounds
    like the scalar one, and both kernels run the same operations): grids of
    one and several 64-wide tiles, odd and even nx, every boundary pairing,
    each branch."""
    pb = _two_species(nx, ny, bc, react, force)
    p, f0 = _noneq_f(orc, pb)
    out = {}
    for kern in ("generic", "tma_pair"):
        s = D.Solver(pb, "fp32", step_kernel=kern)
        s.set_f(f0)
        s.step(6)
        out[kern] = s.get_f().cpu().numpy()
        assert s.status()[0] == 0
    assert np.array_equal(out["tma_pair"], out["generic"])


def test_step_tile_choice(D):
    """The handle's tile: two cells per thread for two species on grids of
    at least 4096 tiles of 64 x 8 cells (or when asked for), else one cell
    per thread; one cell per thread for three and four species, the
    species-staged 64 x 8 two-cell tile for five or more (and for two to
    four when asked for); no tile for the generic, FP64 and BF16DEV
    steps."""
    kh = W.kh_shear_layer(2048, ny=1024)
    small = W.kh_shear_layer(1024)
    cases = [(kh, "fp32", "auto", (64, 8, 2)), (kh, "fp32", "tma_cell", (32, 7, 1)),
             (small, "fp32", "auto", (32, 7, 1)), (small, "fp32", "tma_pair", (64, 8, 2)),
             (small, "fp32", "generic", (0, 0, 0)), (small, "fp64", "auto", (0, 0, 0)),
             (small, "bf16dev", "auto", (0, 0, 0)),
             (W.random_smooth(70, 23, 3), "fp32", "auto", (32, 8, 1)),
             (W.random_smooth(70, 23, 4), "fp32", "tma", (32, 6, 1)),
             (W.random_smooth(70, 23, 3), "fp32", "tma_cell", (32, 8, 1)),
             (W.random_smooth(70, 23, 4), "fp32", "tma_pair", (64, 8, 2)),
             (W.random_smooth(70, 23, 6), "fp32", "auto", (64, 8, 2)),
             (small, "fp32", "tma_staged", (64, 8, 2)),
             (W.random_smooth(70, 23, 1), "fp32", "tma", (64, 4, 1))]
    for pb, prec, kern, want in cases:
        s = D.Solver(pb, prec, step_kernel=kern)
        assert s.step_tile() == want, (pb.name, prec, kern)
        s.close()
    s = D.Solver(W.random_smooth(70, 23, 3), "fp32", step_kernel="tma", thermo="fp64")
    assert s.step_tile() == (32, 8, 1)
    s.close()


@pytest.mark.parametrize("nx,ny,ns,bc", [(45, 17, 3, (W.PERIODIC, W.OUTFLOW)),
                                          (130, 19, 3, (W.OUTFLOW, W.PERIODIC)),
                                          (2, 3, 3, (W.PERIODIC, W.PERIODIC)),
                                          (129, 8, 2, (W.OUTFLOW, W.OUTFLOW)),
                                          (1, 1, 2, (W.PERIODIC, W.PERIODIC)),
                                          (37, 13, 4, (W.PERIODIC, W.OUTFLOW)),
                                          (64, 16, 4, (W.OUTFLOW, W.OUTFLOW)),
                                          (67, 9, 5, (W.PERIODIC, W.PERIODIC)),
                                          (33, 11, 6, (W.OUTFLOW, W.PERIODIC)),
                                          (65, 10, 8, (W.PERIODIC, W.OUTFLOW)),
                                          (3, 2, 8, (W.OUTFLOW, W.OUTFLOW))])
def test_staged_kernel_matches_generic_bitwise(D, orc, nx, ny, ns, bc):
    """The species-staged kernel (each species copied into shared memory for
    its moment sums and again for its update, two buffers, two cells per
    thread) against the generic kernel after 6 FP32 steps, bit for bit, and
    against the one-cell TMA kernel where that exists (S <= 4): grids of one
    and several 64 x 8 tiles with ragged tails, odd nx, grids smaller than
    the stencil, every boundary pairing, reaction (three species) and force
    (two and four or more)."""
    pb = W.random_smooth(nx, ny, ns, seed=23 + ns, reactive=ns == 3, force=ns != 3, bc=bc)
    p, f0 = _noneq_f(orc, pb)
    kerns = ("generic", "tma_staged") + (("tma_cell",) if ns <= 4 else ())
    out = {}
    for kern in kerns:
        s = D.Solver(pb, "fp32", step_kernel=kern)
        if kern == "tma_staged":
            assert s.step_tile() == (64, 8, 2)
        s.set_f(f0)
        s.step(6)
        out[kern] = s.get_f().cpu().numpy()
        assert s.status()[0] == 0, kern
        s.close()
    for kern in kerns[1:]:
        assert np.array_equal(out[kern], out["generic"]), kern


# ---------------------------------------------------------------------------
# Full-size workloads: sampled windows of one step at the bench sizes
# ---------------------------------------------------------------------------

def _windows(nx, ny, rng, k=4, w=24):
    out = [(0, min(w, nx), 0, min(w, ny)), (max(0, nx - w), nx, max(0, ny - w), ny)]
    for _ in range(k):
        x0 = int(rng.integers(0, max(1, nx - w)))
        y0 = int(rng.integers(0, max(1, ny - w)))
        out.append((x0, min(nx, x0 + w), y0, min(ny, y0 + w)))
    return out


@pytest.mark.parametrize("which,prec", [("kh4096", "fp32"), ("reactive1024", "fp32"), ("reactive1024", "fp64")])
def test_full_size_one_step_sampled(D, orc, which, prec):
    pb = W.kh_shear_layer(4096) if which == "kh4096" else W.reactive_premixed()
    s = D.Solver(pb, prec)
    s.set_state()
    f0 = s.get_f()
    s.step(1)
    f1 = s.get_f()
    assert s.status()[0] == 0
    p = orc.params_of(pb)
    f0n = f0.cpu().numpy()
    f1n = f1.cpu().numpy()
    del f0, f1
    rng = np.random.default_rng(0)
    for (x0, x1, y0, y1) in _windows(pb.nx, pb.ny, rng):
        want, st = orc.step_region(p, f0n, x0, x1, y0, y1)
        got = f1n[:, :, y0:y1, x0:x1]
        assert rel_linf(got, want) <= (1e-12 if prec == "fp64" else 1e-6), (x0, y0)


@pytest.mark.parametrize("nx,ny,ns,bc", [(130, 19, 1, (W.PERIODIC, W.PERIODIC)),
                                          (67, 9, 2, (W.OUTFLOW, W.PERIODIC)),
                                          (45, 17, 3, (W.PERIODIC, W.OUTFLOW)),
                                          (1, 1, 2, (W.PERIODIC, W.PERIODIC)),
                                          (33, 21, 2, (W.PERIODIC, W.OUTFLOW)),
                                          (33, 21, 2, (W.OUTFLOW, W.PERIODIC)),
                                          (2, 3, 3, (W.PERIODIC, W.PERIODIC)),
                                          (34, 9, 1, (W.OUTFLOW, W.OUTFLOW)),
                                          (65, 17, 3, (W.PERIODIC, W.PERIODIC)),
                                          (65, 5, 1, (W.PERIODIC, W.OUTFLOW)),
                                          (33, 8, 2, (W.OUTFLOW, W.OUTFLOW)),
                                          (37, 13, 4, (W.PERIODIC, W.OUTFLOW)),
                                          (3, 2, 4, (W.PERIODIC, W.PERIODIC))])
def test_tma_kernel_matches_generic_bitwise(D, orc, nx, ny, ns, bc):
    """The TMA-staged kernel reads its stencil from shared memory and runs
    the same explicitly rounded arithmetic as the generic kernel (two cells
    per thread in packed FP32x2 for two species, one otherwise), so after 6
    FP32 steps the two states are equal bit for bit.  The generic kernel
    reads the stored ghost cells; the TMA kernel writes none and builds a
    boundary tile's halo from the interior, so grids one cell past a tile
    edge, grids smaller than the stencil and every boundary pairing are
    covered."""
    pb = W.random_smooth(nx, ny, ns, seed=21, reactive=ns == 3, force=ns == 2, bc=bc)
    p, f0 = _noneq_f(orc, pb)
    out = {}
    for kern in ("generic", "tma"):
        s = D.Solver(pb, "fp32", step_kernel=kern)
        s.set_f(f0)
        s.step(6)
        out[kern] = s.get_f().cpu().numpy()
        assert s.status()[0] == 0
    assert np.array_equal(out["tma"], out["generic"])


# ---------------------------------------------------------------------------
# BF16-deviation storage
#
# Tolerance: delta = f - f^eq(previous moments) is stored with an 8-bit
# mantissa, a relative rounding of 2^-9 of |delta| per step; for the 5 %
# nonequilibrium states below |delta| <= ~0.1 |f|, so each step adds
# <= 2e-4 |f| of unbiased rounding that the relaxation damps; after 20 steps
# the state stays within 2e-3 of the FP64 oracle (f and moments).
# ---------------------------------------------------------------------------

BF16_TOL = 2e-3


@pytest.mark.parametrize("nx,ny,ns,bc", [(70, 23, 2, (W.OUTFLOW, W.PERIODIC)),
                                          (33, 17, 3, (W.PERIODIC, W.OUTFLOW)),
                                          (9, 5, 1, (W.PERIODIC, W.PERIODIC))])
def test_bf16dev_against_oracle(D, orc, nx, ny, ns, bc):
    pb = W.random_smooth(nx, ny, ns, seed=41, bc=bc)
    p, f0 = _noneq_f(orc, pb)
    s = D.Solver(pb, "bf16dev")
    s.set_f(f0)
    s.step(20)
    f = s.get_f().cpu().numpy()
    mom = s.moments().cpu().numpy()
    assert s.status()[0] == 0
    fr, _ = orc.run(p, f0, 20)
    mr = orc.moments(p, fr)
    assert rel_linf(f, fr) <= BF16_TOL
    errs = moments_errors(mom, mr, pb.ns)
    assert np.all(errs <= BF16_TOL), errs


def test_bf16dev_set_state_is_the_equilibrium(D, orc):
    pb = W.random_smooth(29, 13, 2, seed=5)
    s = D.Solver(pb, "bf16dev")
    s.set_state()
    p, f0 = _oracle_f0(orc, pb)
    # zero deviation: f is the FP32 equilibrium of the stored FP32 moments.
    # Rounding n, u and T to float (6e-8 relative each) and forming T/m in
    # float moves the equilibrium by up to ~20x that (the D2V16 f^eq weighs
    # T^2 and u^4 terms against each other), so the bound is 2e-6.
    assert rel_linf(s.get_f().cpu().numpy(), f0) <= 2e-6


def test_bf16dev_conservation(D, orc):
    pb = W.random_smooth(64, 64, 2, seed=13)
    s = D.Solver(pb, "bf16dev")
    s.set_state()
    c0 = s.conservation().cpu().numpy()
    s.step(200)
    c1 = s.conservation().cpu().numpy()
    assert np.max(np.abs(c1[:2] - c0[:2]) / np.abs(c0[:2])) < 1e-5
    assert abs(c1[4] - c0[4]) / abs(c0[4]) < 1e-5


@pytest.mark.parametrize("prec,ns", [("fp32", 2), ("fp32", 1), ("fp64", 3), ("bf16dev", 2)])
def test_page_locked_host_fields(D, prec, ns):
    """dbm_set_state from page-locked host fields, and dbm_moments,
    dbm_conservation and dbm_get_f into page-locked host memory, give the
    bits of the same calls on device arrays: staged through the free state
    buffer where it is large enough (two species FP32, FP64), read or
    written in place otherwise (one species FP32 moments, BF16DEV moments);
    the staging leaves the state alone (the runs stay equal step after
    step)."""
    pb = W.random_smooth(45, 19, ns, seed=8)
    a, b = D.Solver(pb, prec), D.Solver(pb, prec)
    fields = [np.ascontiguousarray(x, dtype=np.float64) for x in (pb.rho_s, pb.ux, pb.uy, pb.T)]
    dev = [torch.from_numpy(x).to(a.device) for x in fields]
    host = [torch.from_numpy(x.copy()).pin_memory() for x in fields]
    D.dbm_set_state(a.h, *[t.data_ptr() for t in dev], a._st())
    D.dbm_set_state(b.h, *[t.data_ptr() for t in host], b._st())
    for rnd in range(2):
        a.step(3)
        b.step(3)
        ma = a.moments().cpu().numpy()
        mh = torch.empty(ma.shape, dtype=torch.float64).pin_memory()
        D.dbm_moments(b.h, mh.data_ptr(), b._st())
        ca = a.conservation().cpu().numpy()
        ch = torch.empty(ca.shape, dtype=torch.float64).pin_memory()
        D.dbm_conservation(b.h, ch.data_ptr(), b._st())
        fa = a.get_f().cpu().numpy()
        fh = torch.empty(fa.shape, dtype=torch.float64).pin_memory()
        D.dbm_get_f(b.h, fh.data_ptr(), b._st())
        torch.cuda.synchronize()
        assert np.array_equal(mh.numpy(), ma), rnd
        assert np.array_equal(ch.numpy(), ca), rnd
        assert np.array_equal(fh.numpy(), fa), rnd
    assert a.status() == (0, 0) and b.status() == (0, 0)
    a.close()
    b.close()
