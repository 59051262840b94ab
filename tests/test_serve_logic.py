"""Host-side logic of the serving layer: admission, quanta, the request mix
and the sequential-service reference (no GPU)."""
import math

import numpy as np
import pytest

from paper_2006_15932_gb300 import workloads as W

torch = pytest.importorskip("torch")
serve = pytest.importorskip("paper_2006_15932_gb300.serve")


def test_admission_never_exceeds_budget():
    a = serve.Admission(100)
    assert a.fits(60)
    a.admit(60)
    assert not a.fits(41) and a.fits(40)
    a.admit(40)
    assert a.used == 100 and a.peak == 100
    a.release(60)
    assert a.fits(60) and not a.fits(61)
    with pytest.raises(AssertionError):
        a.admit(61)


def test_quantum_never_oversteps_a_member():
    assert serve.quantum([500, 130, 900], 128) == 128
    assert serve.quantum([500, 100, 900], 128) == 100
    assert serve.quantum([1], 128) == 1
    # stepping every member by the quantum, repeatedly, lands each exactly
    rem = [7, 300, 129, 128]
    steps = [0] * 4
    while rem:
        q = serve.quantum(rem, 128)
        steps = [s + q for s in steps]
        rem = [r - q for r in rem]
        assert min(rem) >= 0
        rem = [r for r in rem if r > 0]
    # (the remaining counts all reach zero without going negative)


def test_sequential_reference_by_hand():
    specs = [W.RequestSpec(rid=0, kind="shock", L=10, ns=2, seed=0, nsteps=10, arrival=0.0),   # 2000 units
             W.RequestSpec(rid=1, kind="shock", L=10, ns=4, seed=0, nsteps=10, arrival=1.0),   # 4000 units
             W.RequestSpec(rid=2, kind="shock", L=10, ns=2, seed=0, nsteps=5, arrival=10.0)]   # 1000 units
    r = serve.simulate_sequential(specs, {2: 1000.0, 4: 1000.0})
    # finishes: 2.0, 6.0, 11.0 -> latencies 2, 5, 1
    assert r["makespan_s"] == pytest.approx(11.0)
    assert r["mean_s"] == pytest.approx((2 + 5 + 1) / 3)
    assert r["throughput"] == pytest.approx(7000 / 11.0)


def test_serving_mix_follows_its_recipe():
    specs = W.serving_requests(300, seed=5)
    assert len(specs) == 300
    L = np.array([s.L for s in specs])
    assert L.min() >= 128 and L.max() <= 2048
    # log-uniform sides: the median sits near the geometric mean of 128 and 2048
    assert abs(math.log(np.median(L)) - 0.5 * math.log(128 * 2048)) < 0.25
    assert {s.ns for s in specs} == {2, 3, 4}
    steps = np.array([s.nsteps for s in specs])
    assert steps.min() >= 1000 and steps.max() <= 10000
    frac = np.mean([s.kind == "reactive" for s in specs])
    assert 0.4 < frac < 0.6
    again = W.serving_requests(300, seed=5)
    assert [(s.L, s.ns, s.kind, s.nsteps, s.seed) for s in specs] == [(s.L, s.ns, s.kind, s.nsteps, s.seed)
                                                                        for s in again]


def test_poisson_arrivals():
    specs = W.poisson_arrivals(W.serving_requests(2000, seed=2, hi=256), rate=50.0)
    t = np.array([s.arrival for s in specs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 50.0) < 0.1 / 50.0
    # exponential gaps: the coefficient of variation is one
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1


@pytest.mark.parametrize("kind,ns", [("shock", 2), ("shock", 4), ("reactive", 2), ("reactive", 3), ("reactive", 4)])
def test_request_fields_and_problem(kind, ns):
    spec = W.RequestSpec(rid=3, kind=kind, L=48, ns=ns, seed=11, nsteps=5)
    pb = W.request_problem(spec)
    assert pb.ns == ns and pb.nx == pb.ny == 48
    rho_s, ux, uy, T = W.request_fields(spec)
    assert rho_s.shape == (ns, 48, 48) and ux.shape == (48, 48)
    assert torch.all(rho_s >= 0) and torch.all(T > 0)
    if kind == "reactive":
        assert pb.k_ov > 0
        # the one-step reaction conserves mass: sum a m = 0
        assert sum(s.a * s.m for s in pb.species) == pytest.approx(0.0, abs=1e-15)
        assert pb.species[pb.fuel].a < 0 and pb.species[pb.oxid].a < 0
        assert torch.allclose(rho_s.sum(0), torch.ones(48, 48, dtype=torch.float64))
    else:
        rho = rho_s.sum(0)
        assert set(torch.unique(rho).tolist()) == {0.125, 1.0}
        assert torch.allclose(rho * T, torch.where(rho > 0.5, 1.0, 0.1).to(torch.float64))


def test_summary_leaves_out_withdrawn_requests():
    mk = lambda rid, fin, cancelled=False: serve.Result(rid=rid, ns=2, cells=100, nsteps=10, arrival=0.0,
                                                        admitted=0.0, finished=fin, status=0,
                                                        conservation=np.zeros(6), cancelled=cancelled)
    rs = [mk(0, 1.0), mk(1, 3.0), mk(2, 0.1, cancelled=True)]
    d = serve.summarize(rs)
    assert d["requests"] == 2 and d["units"] == 2 * 2000
    assert d["makespan_s"] == 3.0 and d["p50_s"] == 2.0
