"""Failure detection without a GPU fault.  Every wait of the particle
launches is bounded in time; a wait that runs out sets PIC_STATUS_TIMEOUT and
lets the launch end.  The self-test entry runs that very wait on a barrier
that nothing completes (no copy is issued, so no memory is ever written and
nothing can fault): it must give up at its limit, report the status, and
leave the context usable for the next run."""
import ctypes

import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("limit_ms", [5, 50])
def test_bounded_wait_runs_out_reports_and_context_stays_usable(limit_ms):
    from paper_1310_5284_gb300 import _abi
    from paper_1310_5284_gb300.sim import Sim

    st, waited = ctypes.c_uint32(0), ctypes.c_double(0.0)
    r = _abi.lib().pic_selftest_wait(limit_ms * 1_000_000, ctypes.byref(st), ctypes.byref(waited), None)
    assert r == -6  # PIC_ETIMEOUT
    assert st.value == _abi.PIC_STATUS_TIMEOUT
    assert limit_ms * 1e-3 <= waited.value < limit_ms * 1e-3 + 0.5
    sim = Sim(dict(workloads.CFG_SMALL_CCP, np_init=4000), device="cuda:0")
    sim.step(3)
    assert sim.status() == 0 and sim.diag()["step"] == 3
    sim.close()
