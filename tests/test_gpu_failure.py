"""Failure detection on the GPU without a fault: the two waits that every
reduction kernel bounds (the decoupled look-back on a predecessor tile's
state, and the wait for a TMA block's mbarrier phase) are made to run out,
on a state that nothing publishes and a phase that nothing completes.  Each
must give up at its bound and report SEMR_STATUS_TIMEOUT; the barrier wait is
followed, as in the reduce kernel's abort path, by a second bounded wait for
a copy that could still land, which gives up too and adds SEMR_STATUS_STAGE.
The context must stay usable.  Nothing traps, faults or spins without a
limit."""
import time

import pytest

import oracle
import paper_2407_20731_b300 as semr
from parity import compare_payloads, make_case, run_gpu

pytestmark = pytest.mark.gpu


def test_bounded_waits_time_out_and_report():
    t0 = time.perf_counter()
    st_lookback, st_barrier = semr.semr_selftest_waits()
    elapsed = time.perf_counter() - t0
    assert st_lookback == semr.SEMR_STATUS_TIMEOUT
    assert st_barrier == semr.SEMR_STATUS_TIMEOUT | semr.SEMR_STATUS_STAGE
    assert elapsed < 30.0, elapsed
    # the context is still usable: a reduction right after is bit-exact with the oracle
    fields, jac = make_case(300, 8, 1, seed=3)
    res, _ = run_gpu(fields, jac, 8, 1e-3)
    assert res.summary.status == 0
    o = oracle.reduce(fields.cpu().numpy(), jac.cpu().numpy(), 1e-3, fragile_cap=10000)
    compare_payloads(res.payload, o.payload, o.fragile)
