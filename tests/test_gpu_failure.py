"""Failure detection on the GPU without a GPU fault: a bounded device wait
that runs out (the bulk-copy kernels' poll loop on an mbarrier that nothing
completes, tetm_rz_selftest_wait) reports TETM_E_TIMEOUT through the device
error word, the context stays usable, and the kernels' own limit gives up
within seconds."""
import time

import numpy as np
import pytest

from oracle import RzOracle
from paper_0901_1053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MAX_POLLS = 1 << 18   # TETM_RZ_MAX_POLLS, include/tetm_rz.h


@pytest.fixture(scope="module")
def tetm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_1053_gb300 import tetm as t
    return t


def test_bounded_wait_times_out_and_the_context_stays_usable(tetm):
    t0 = time.perf_counter()
    rc_short = tetm.rz_selftest_wait(1000)
    t1 = time.perf_counter()
    rc_long = tetm.rz_selftest_wait(200000)
    t2 = time.perf_counter()
    assert rc_short == tetm.TETM_E_TIMEOUT
    assert rc_long == tetm.TETM_E_TIMEOUT
    per_poll = max((t2 - t1) - (t1 - t0), 0.0) / 199000
    assert per_poll * MAX_POLLS < 5.0, per_poll    # the step kernels give up within seconds
    # the context still solves correctly
    w = wl.cavity_chain_rz(24, 60, 0, 1, sigma_cells=2.5, precision="fp64", n_cells=2, i0=3)
    s = tetm.RzSolver(w.nr, w.nz, w.m_lo, w.m_hi, w.dr, w.dz, w.cdt, "fp64", pec=w.pec)
    s.set_kernel("bulk")
    s.set_bunch(w.sigma, w.charge, w.i0)
    s.step(w.steps)
    s.sync()
    for m in (0, 1):
        o = RzOracle(w.nr, w.nz, m, w.dr, w.dz, w.cdt, pec=w.pec)
        o.set_bunch(w.sigma, w.charge, w.i0)
        o.step(w.steps)
        ref = o.wake()[0]
        assert np.max(np.abs(s.wake(m)[0] - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_selftest_arguments(tetm):
    assert tetm.rz_selftest_wait(0) == tetm.TETM_E_ARG
    assert tetm.rz_selftest_wait(1 << 27) == tetm.TETM_E_ARG
