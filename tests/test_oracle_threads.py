"""The oracle's thread count (set for timing it on one core and on all of
them) changes nothing in its results: its OpenMP loop runs over rows, each
row's cells are computed from the old field alone, and the status bits are
OR-reduced."""
import numpy as np

from paper_2006_15932_gb300 import workloads as W


def test_thread_count_does_not_change_results(orc):
    pb = W.random_smooth(40, 23, 3, seed=17, reactive=True, force=True, bc=(W.OUTFLOW, W.PERIODIC))
    p = orc.params_of(pb)
    f0 = orc.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)
    all_threads = orc.set_threads(0)
    try:
        out = {}
        for n in (1, max(2, all_threads)):
            assert orc.set_threads(n) == n
            out[n] = orc.run(p, f0, 3)
        (fa, sa), (fb, sb) = out.values()
        assert sa == sb == 0
        assert np.array_equal(fa, fb)
    finally:
        orc.set_threads(all_threads)
