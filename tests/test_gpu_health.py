"""Failure detection on the GPU without a fault: every bounded wait of the
TMA-staged steps reports through the health flag when it gives up.

A handle made with dbm_params.wait_polls < 0 polls its first tile copy zero
times before giving up, so each CTA takes the timeout path at once: it
raises DBM_HEALTH_TIMEOUT, then waits (bounded, with the full limit) for its
copy, which is valid and lands; the all-species kernels then leave without
writing, the species-staged kernel goes on with its step.  Nothing faults
or hangs; the descriptor and buffers stay valid.  The status call must report
DBM_ERR_TIMEOUT with bit 16, and a normal solve afterwards in the same
context must be green and correct.
"""
import numpy as np
import pytest

from paper_2006_15932_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT_RC, TIMEOUT_BIT = -8, 16


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_15932_gb300 import build as B
    from paper_2006_15932_gb300 import dbm

    B.build()
    dbm.load()
    return dbm


@pytest.mark.parametrize("ns,kernel", [(2, "tma_cell"), (2, "tma_pair"), (3, "tma"), (3, "tma_staged"),
                                       (2, "tma_staged"), (5, "tma")])
def test_tile_wait_timeout_is_reported(D, orc, ns, kernel):
    pb = W.random_smooth(70, 20, ns, seed=5, reactive=ns == 3)
    s = D.Solver(pb, "fp32", step_kernel=kernel, wait_polls=-1)
    assert s.step_tile()[0] > 0  # a TMA-staged step
    s.set_state()
    s.step(2)
    rc, bits = s.status()
    assert rc == TIMEOUT_RC and bits & TIMEOUT_BIT, (rc, bits)
    assert "timed out" in D.dbm_last_error(s.h)
    s.close()
    # the context is still usable: the same problem without the knob is
    # green and matches the oracle
    ok = D.Solver(pb, "fp32", step_kernel=kernel)
    ok.set_state()
    ok.step(3)
    assert ok.status() == (0, 0)
    p = orc.params_of(pb)
    ref, st = orc.run(p, orc.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T), 3)
    assert st == 0
    f = ok.get_f().cpu().numpy()
    assert np.max(np.abs(f - ref)) / np.max(np.abs(ref)) <= 2e-5
    ok.close()


def test_batched_tile_wait_timeout_is_reported(D):
    """The batched kernel reads each instance's wait limit from its own
    block: only the instances made with the knob report the timeout, and
    the persistent form leaves after its first tile."""
    stream = torch.cuda.Stream()
    pbs = [W.shock_instance(40, 1), W.reactive_instance(36, 2), W.shock_instance(48, 3)]
    polls = [-1, 0, -1]
    sols = []
    for q, wp in zip(pbs, polls):
        sols.append(D.Solver(q, "fp32", stream=stream, wait_polls=wp))
        sols[-1].set_state()
    for persistent in (0, 1):
        for s_ in sols:
            s_.set_state()
        batch = D.Batch(sols, stream=stream, config={"tile": (32, 8), "persistent": persistent, "promote": 1})
        batch.step(3)
        got = [s_.status() for s_ in sols]
        for (rc, bits), wp in zip(got, polls):
            if wp < 0:
                assert rc == TIMEOUT_RC and bits & TIMEOUT_BIT, (persistent, got)
            else:
                assert (rc, bits) == (0, 0), (persistent, got)
        batch.close()
    for s_ in sols:
        s_.close()
