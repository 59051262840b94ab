"""dbm_conservation_noalloc: the conserved totals for callers that cannot
allocate device memory (for example a plug-in inside a host application
that owns all of the GPU's memory), so cannot give the library a scratch
buffer.  Its reduction partials live in a static device array inside the
library.  Checked through the C ABI against dbm_conservation, which uses
the caller's scratch buffer, on two calls in a row.

This file is collected last on purpose, so that a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2006_15932_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12  # the FP64 tolerance of the other output tests


@pytest.fixture(scope="module")
def D():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_15932_gb300 import build as B
    from paper_2006_15932_gb300 import dbm

    B.build()
    dbm.load()
    return dbm


@pytest.mark.parametrize("prec,ns", [("fp64", 2), ("fp32", 3), ("fp32", 4), ("bf16dev", 2)])
def test_noalloc_totals_match_scratch_version(D, prec, ns):
    pb = W.random_smooth(53, 21, ns, seed=31, reactive=ns >= 3 and prec != "bf16dev")
    s = D.Solver(pb, prec)
    s.set_state()
    for call in range(2):
        ref = s.conservation()
        out = torch.full((ns + 4,), float("nan"), dtype=torch.float64, device=s.device)
        # call 0: the handle's current state; call 1: the same state by pointer
        cur = D.dbm_steps_taken(s.h) % 2
        state = 0 if call == 0 else s.buf[cur].data_ptr()
        D.dbm_conservation_noalloc(s.h, state, out.data_ptr(), s._st())
        a = out.cpu().numpy()
        b = ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)) <= TOL, (call, a, b)
        s.step(3)
    s.close()


def test_noalloc_rejects_partials_beyond_its_array(D):
    pb = W.random_smooth(8, 8, 5, seed=1)
    s = D.Solver(pb, "fp32")
    s.set_state()
    out = torch.empty(9, dtype=torch.float64, device=s.device)
    with pytest.raises(D.DbmError) as e:
        D.dbm_conservation_noalloc(s.h, 0, out.data_ptr(), s._st())
    assert e.value.code == -1 and "static scratch" in str(e.value)
    s.close()
