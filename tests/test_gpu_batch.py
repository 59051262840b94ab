"""Batched stepping (dbm_batch_*): many independent FP32 problems advanced
by one persistent launch per step, replayed from CUDA graphs."""
import numpy as np
import pytest

from paper_2006_15932_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_15932_gb300 import build as B
    from paper_2006_15932_gb300 import dbm

    B.build()
    dbm.load()
    return dbm


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _mixed(n=8, seed=3):
    return W.batched_instances(n, seed=seed, lo=21, hi=140)


def test_batch_matches_individual_steps(D):
    pbs = _mixed()
    stream = torch.cuda.Stream()
    solo, mixed = [], []
    for pb in pbs:
        for group in (solo, mixed):
            s = D.Solver(pb, "fp32", stream=stream)
            s.set_state()
            group.append(s)
    for s in solo:
        s.step(21)
    batch = D.Batch(mixed, stream=stream)
    batch.step(21)  # 10 graph pairs + 1 single step
    torch.cuda.synchronize()
    for a, b in zip(solo, mixed):
        assert b.status()[0] == 0
        assert D.dbm_steps_taken(b.h) == 21
        fa, fb = a.get_f().cpu().numpy(), b.get_f().cpu().numpy()
        assert np.array_equal(fb, fa)  # the same explicitly rounded arithmetic


def test_batch_tune_leaves_states_unchanged(D):
    pbs = _mixed(6, seed=5)
    stream = torch.cuda.Stream()
    sols = []
    for pb in pbs:
        s = D.Solver(pb, "fp32", stream=stream)
        s.set_state()
        s.step(3)
        sols.append(s)
    before = [s.get_f().cpu().numpy() for s in sols]
    batch = D.Batch(sols, stream=stream, tune=True)
    info = batch.info()
    assert info["tile"] in ((32, 10), (32, 8), (32, 16), (32, 7), (64, 4), (64, 8)) and info["tiles"] > 0
    cfg = batch.config()
    assert (cfg["tile"], cfg["cells"]) in (((32, 10), 1), ((32, 8), 1), ((32, 16), 1), ((32, 7), 1), ((64, 4), 1),
                                           ((64, 8), 2), ((32, 16), 2))
    after = [s.get_f().cpu().numpy() for s in sols]
    for a, b in zip(before, after):
        assert np.array_equal(a, b)


def test_batch_against_oracle(D, orc):
    pbs = [W.shock_instance(24, 1), W.reactive_instance(19, 2), W.shock_instance(33, 3)]
    stream = torch.cuda.Stream()
    sols = []
    for pb in pbs:
        s = D.Solver(pb, "fp32", stream=stream)
        s.set_state()
        sols.append(s)
    batch = D.Batch(sols, stream=stream)
    batch.step(30)
    torch.cuda.synchronize()
    for pb, s in zip(pbs, sols):
        p = orc.params_of(pb)
        f0 = orc.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)
        fr, st = orc.run(p, f0, 30)
        assert st == 0
        assert rel(s.get_f().cpu().numpy(), fr) <= 2e-5


def test_batch_picks_up_a_reset_handle(D):
    pbs = _mixed(4, seed=9)
    stream = torch.cuda.Stream()
    sols, ref = [], []
    for pb in pbs:
        for group in (sols, ref):
            s = D.Solver(pb, "fp32", stream=stream)
            s.set_state()
            group.append(s)
    batch = D.Batch(sols, stream=stream, tune=False)
    batch.step(5)
    sols[1].set_state()  # restart one instance from its initial fields
    batch.step(4)
    for k, s in enumerate(ref):
        s.step(4 if k == 1 else 9)
    torch.cuda.synchronize()
    for a, b in zip(ref, sols):
        assert np.array_equal(b.get_f().cpu().numpy(), a.get_f().cpu().numpy())


def test_batch_rejects_mixed_species_or_precision(D):
    stream = torch.cuda.Stream()
    a = D.Solver(W.random_smooth(16, 8, 2), "fp32", stream=stream)
    b = D.Solver(W.random_smooth(16, 8, 3), "fp32", stream=stream)
    c = D.Solver(W.random_smooth(16, 8, 2), "fp64", stream=stream)
    for group in ([a, b], [a, c]):
        with pytest.raises(D.DbmError):
            D.Batch(group, stream=stream)


@pytest.mark.parametrize("ns,n", [(1, 131), (2, 130), (3, 126), (4, 124)])
def test_batch_spanning_several_launch_chunks(D, ns, n):
    """More instances than one launch's parameter block holds (125, 123, 122
    and 121 instances for S = 1, 2, 3, 4): the batch runs several chunks per
    step; every instance must still match its own single-problem steps."""
    rng = np.random.default_rng(40 + ns)
    pbs = []
    for k in range(n):
        nx, ny = int(rng.integers(5, 41)), int(rng.integers(3, 29))
        bc = (k % 2, (k // 2) % 2)
        pbs.append(W.random_smooth(nx, ny, ns, seed=100 * ns + k, reactive=(ns >= 3 and k % 2 == 0),
                                   force=(k % 4 == 1), bc=bc))
    stream = torch.cuda.Stream()
    solo, mixed = [], []
    for pb in pbs:
        for group in (solo, mixed):
            s = D.Solver(pb, "fp32", stream=stream)
            s.set_state()
            group.append(s)
    for s in solo:
        s.step(7)
    batch = D.Batch(mixed, stream=stream, tune=(ns == 2))
    batch.step(7)  # three graph pairs and one single step
    torch.cuda.synchronize()
    # same per-cell arithmetic, compiled into different kernels (the
    # compiler may contract different products); the force term's
    # difference of two equilibria amplifies those last-bit differences
    for a, b in zip(solo, mixed):
        assert b.status()[0] == 0
        assert rel(b.get_f().cpu().numpy(), a.get_f().cpu().numpy()) <= 4e-6


def test_batch_on_the_default_stream(D):
    """Without a created stream the steps are launched one by one."""
    pbs = _mixed(5, seed=21)
    solo, mixed = [], []
    for pb in pbs:
        for group in (solo, mixed):
            s = D.Solver(pb, "fp32")
            s.set_state()
            group.append(s)
    for s in solo:
        s.step(6)
    batch = D.Batch(mixed, stream=torch.cuda.default_stream(), tune=False)
    batch.step(6)
    torch.cuda.synchronize()
    for a, b in zip(solo, mixed):
        assert np.array_equal(b.get_f().cpu().numpy(), a.get_f().cpu().numpy())


def _two_steps_window(orc, p, f0, x0, x1, y0, y1):
    """Oracle f after two steps on the window [x0,x1) x [y0,y1): the first
    step on the window grown by the stencil radius (wrapped or clamped by the
    oracle's own boundary handling), the second on the window."""
    nx, ny = p.nx, p.ny
    f1 = f0.copy()
    gx0, gx1 = max(0, x0 - 2), min(nx, x1 + 2)
    gy0, gy1 = max(0, y0 - 2), min(ny, y1 + 2)
    # cells within 2 of the window across a periodic edge wrap around: step
    # the whole grid rows / columns in that case (small instances only)
    if p.bc_x == W.PERIODIC and (x0 < 2 or x1 > nx - 2):
        gx0, gx1 = 0, nx
    if p.bc_y == W.PERIODIC and (y0 < 2 or y1 > ny - 2):
        gy0, gy1 = 0, ny
    reg, st = orc.step_region(p, f0, gx0, gx1, gy0, gy1)
    assert st == 0
    f1[:, :, gy0:gy1, gx0:gx1] = reg
    out, st = orc.step_region(p, f1, x0, x1, y0, y1)
    assert st == 0
    return out


def test_batched_workload_full_size_sampled(D, orc):
    """The batched benchmark configuration at full size (64 instances,
    sides 64..512, shock tubes and reactive gases), tuned and stepped by one
    two-step graph replay exactly as the benchmark times it; sampled windows
    of eight instances against the oracle."""
    pbs = W.batched_instances()
    stream = torch.cuda.Stream()
    sols = []
    for pb in pbs:
        s = D.Solver(pb, "fp32", stream=stream)
        s.set_state()
        sols.append(s)
    batch = D.Batch(sols, stream=stream, tune=True)
    f0s = {k: sols[k].get_f().cpu().numpy() for k in range(0, 64, 8)}
    batch.step(2)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    for k, f0 in f0s.items():
        pb = pbs[k]
        assert sols[k].status()[0] == 0
        f2 = sols[k].get_f().cpu().numpy()
        p = orc.params_of(pb)
        w = 16
        corners = [(0, 0), (pb.nx - w, pb.ny - w),
                   (int(rng.integers(0, pb.nx - w)), int(rng.integers(0, pb.ny - w)))]
        for x0, y0 in corners:
            want = _two_steps_window(orc, p, f0, x0, x0 + w, y0, y0 + w)
            got = f2[:, :, y0:y0 + w, x0:x0 + w]
            assert rel(got, want) <= 1e-6, (k, x0, y0)
    batch.close()


SHAPES = [((32, 10), 1), ((32, 8), 1), ((32, 16), 1), ((32, 7), 1), ((64, 4), 1), ((64, 8), 2), ((32, 16), 2)]


@pytest.mark.parametrize("tile,cells", SHAPES)
def test_every_batch_shape_matches_single_problem_steps(D, tile, cells):
    """Each compiled tile shape, one CTA per tile and persistent, gives the
    bits of the single-problem steps on a mix of shock tubes (outflow in x)
    and reactive gases (periodic) whose sides leave ragged tiles."""
    pbs = _mixed(6, seed=31)
    stream = torch.cuda.Stream()
    solo = []
    for pb in pbs:
        s = D.Solver(pb, "fp32", stream=stream)
        s.set_state()
        s.step(5)
        solo.append(s)
    want = [s.get_f().cpu().numpy() for s in solo]
    for persistent in (0, 1):
        mixed = []
        for pb in pbs:
            s = D.Solver(pb, "fp32", stream=stream)
            s.set_state()
            mixed.append(s)
        batch = D.Batch(mixed, stream=stream, config={"tile": tile, "cells": cells, "persistent": persistent,
                                                      "promote": 1})
        assert batch.config()["cells"] == cells and batch.config()["tile"] == tile
        batch.step(5)
        torch.cuda.synchronize()
        for a, b in zip(want, mixed):
            assert b.status()[0] == 0
            assert np.array_equal(b.get_f().cpu().numpy(), a)
        batch.close()
