"""Serving (continuous batching) on the GPU: results do not depend on the
mix a request is served in, admission respects the HBM budget, and every
request gets exactly its own number of steps."""
import numpy as np
import pytest

from paper_2006_15932_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_15932_gb300 import build as B
    from paper_2006_15932_gb300 import dbm, serve

    B.build()
    dbm.load()
    return serve


def _mix():
    rng = np.random.default_rng(7)
    specs = []
    for k in range(9):
        specs.append(W.RequestSpec(rid=k, kind="reactive" if k % 2 else "shock", L=int(rng.integers(30, 90)),
                                   ns=(2, 3, 4)[k % 3], seed=1000 + k, nsteps=int(rng.integers(9, 40)),
                                   arrival=0.01 * k))
    return specs


def _alone(S, spec):
    srv = S.Server(qmax=8, keep_f=True, hbm_budget=1 << 32)
    spec0 = W.RequestSpec(**{**spec.__dict__, "arrival": 0.0})
    (r,) = srv.run([spec0])
    return r


def test_same_result_alone_and_in_the_mix(S):
    from paper_2006_15932_gb300 import dbm as D

    specs = _mix()
    srv = S.Server(qmax=8, keep_f=True, hbm_budget=1 << 32)
    res = {r.rid: r for r in srv.run(specs)}
    assert sorted(res) == [s.rid for s in specs]
    assert all(r.status == 0 for r in res.values())
    # several quanta, several rebuilds: the mix really changed under the requests
    assert sum(g.rebuilds for g in srv.groups.values()) >= 3
    for spec in specs:
        alone = _alone(S, spec)
        np.testing.assert_array_equal(alone.f, res[spec.rid].f)
        np.testing.assert_array_equal(alone.conservation, res[spec.rid].conservation)
    # and the served result is the plain FP32 solve of the same problem
    for spec in specs[:3]:
        s = D.Solver(W.request_problem(spec), "fp32")
        s.set_state(*W.request_fields(spec, "cuda"))
        s.step(spec.nsteps)
        f = s.get_f().cpu().numpy()
        np.testing.assert_array_equal(f, res[spec.rid].f)  # the same explicitly rounded arithmetic


def test_admission_respects_the_hbm_budget(S):
    specs = [W.RequestSpec(rid=k, kind="shock", L=64, ns=2, seed=k, nsteps=20, arrival=0.0) for k in range(6)]
    one = S.footprint(W.request_problem(specs[0]))
    srv = S.Server(qmax=4, hbm_budget=int(2.5 * one))
    res = srv.run(specs)
    assert len(res) == 6 and all(r.status == 0 for r in res)
    assert srv.adm.peak <= srv.adm.budget and srv.adm.peak == 2 * one
    assert srv.adm.used == 0
    # first come, first served: admission times follow the request order
    adm = [r.admitted for r in sorted(res, key=lambda r: r.rid)]
    assert adm == sorted(adm)


def test_request_larger_than_the_budget_is_refused(S):
    spec = W.RequestSpec(rid=0, kind="shock", L=64, ns=2, seed=0, nsteps=3)
    srv = S.Server(hbm_budget=1000)
    with pytest.raises(ValueError):
        srv.run([spec])


def test_zero_step_request_returns_its_initial_state(S):
    from paper_2006_15932_gb300 import dbm as D

    spec = W.RequestSpec(rid=0, kind="reactive", L=40, ns=3, seed=3, nsteps=0)
    srv = S.Server(keep_f=True, hbm_budget=1 << 32)
    (r,) = srv.run([spec])
    s = D.Solver(W.request_problem(spec), "fp32")
    s.set_state(*W.request_fields(spec, "cuda"))
    np.testing.assert_array_equal(r.f, s.get_f().cpu().numpy())


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _oracle_final(orc, spec):
    pb = W.request_problem(spec)
    rho_s, ux, uy, T = (t.numpy() for t in W.request_fields(spec, "cpu"))
    p = orc.params_of(pb)
    fr, st = orc.run(p, orc.init_feq(p, rho_s, ux, uy, T), spec.nsteps)
    assert st == 0
    return fr


def test_served_results_match_the_oracle(S, orc):
    """Every request of a mix served with continuous batching (shock tubes
    and reactive gases, two to four species, arriving while others run)
    against the FP64 oracle's solve of the same request, at the FP32 bound
    of the parity tests (relative L-inf 2e-5 on f)."""
    specs = [W.RequestSpec(rid=0, kind="shock", L=40, ns=2, seed=11, nsteps=30, arrival=0.0),
             W.RequestSpec(rid=1, kind="reactive", L=36, ns=3, seed=12, nsteps=40, arrival=0.0),
             W.RequestSpec(rid=2, kind="reactive", L=33, ns=4, seed=13, nsteps=25, arrival=0.01),
             W.RequestSpec(rid=3, kind="reactive", L=44, ns=2, seed=14, nsteps=35, arrival=0.02),
             W.RequestSpec(rid=4, kind="shock", L=30, ns=3, seed=15, nsteps=20, arrival=0.03),
             W.RequestSpec(rid=5, kind="shock", L=34, ns=4, seed=16, nsteps=33, arrival=0.03)]
    srv = S.Server(qmax=8, keep_f=True, hbm_budget=1 << 32)
    res = {r.rid: r for r in srv.run(specs)}
    assert sorted(res) == [q.rid for q in specs]
    for spec in specs:
        assert res[spec.rid].status == 0
        err = _rel(res[spec.rid].f, _oracle_final(orc, spec))
        assert err <= 2e-5, (spec, err)


def test_sequential_fp64_baseline_matches_the_oracle(S, orc):
    """The baseline the server is compared with (one request at a time,
    plain FP64 solves) is itself held to the oracle at the FP64 bound."""
    specs = [W.RequestSpec(rid=0, kind="reactive", L=30, ns=3, seed=21, nsteps=15),
             W.RequestSpec(rid=1, kind="shock", L=26, ns=2, seed=22, nsteps=12)]
    res = {r.rid: r for r in S.run_sequential(specs, "fp64", keep_f=True)}
    for spec in specs:
        assert res[spec.rid].status == 0
        assert _rel(res[spec.rid].f, _oracle_final(orc, spec)) <= 1e-12


def test_cancelled_requests_leave_and_the_others_are_unchanged(S):
    """A request withdrawn while it waits leaves at once; one withdrawn while
    it runs leaves its group at the next quantum boundary; their memory is
    returned, and every other request's result is bitwise its result alone."""
    import dataclasses

    specs = _mix()
    specs[8] = dataclasses.replace(specs[8], arrival=5.0, cancel_at=0.001)  # still waiting when withdrawn
    specs[2] = dataclasses.replace(specs[2], nsteps=10 ** 6, cancel_at=0.05)  # running when withdrawn
    srv = S.Server(qmax=8, keep_f=True, hbm_budget=1 << 32)
    res = {r.rid: r for r in srv.run(specs)}
    assert sorted(res) == [s.rid for s in specs]
    assert res[8].cancelled and res[8].admitted is None
    assert res[2].cancelled and res[2].admitted is not None
    assert srv.adm.used == 0
    for spec in specs:
        if spec.rid in (2, 8):
            continue
        r = res[spec.rid]
        assert not r.cancelled and r.status == 0
        np.testing.assert_array_equal(_alone(S, spec).f, r.f)
