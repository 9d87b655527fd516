"""Bounded device-side waits (failure detection without a GPU fault).

The tensor-core kernels never wait without a limit: a wait on an mbarrier that
runs out records a bit in the network's status word, the CTA releases its
tensor memory and returns, and the call reports JET_ETIMEOUT.  The time-out is
made to happen here the way that leaves nothing in flight: jet_selftest_wait
runs one CTA that holds tensor memory and waits, with the same bounded-wait
helper, on an mbarrier that nothing arrives on, then at the chained small
levels' grid barrier (the same helper as that kernel's) for a block that does
not exist.  The call must report the time-out after about twice the requested
limit, and the same handle must then contract normally and match the oracle
(the status word was cleared, the context is intact, the tensor memory was
released)."""
import time

import numpy as np
import pytest

import oracle
from circuits import configs
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_the_handle_stays_usable():
    w = configs.build("grid12")
    net = jet.from_network(w.network, precision="tf32x3", apply_tc_min_kf=1)
    try:
        net.path_greedy(seed=1, n_trials=8)
        before = net.contract(w.outputs)
        for limit_us in (1000, 50000):
            t0 = time.perf_counter()
            with pytest.raises(jet.JetError) as e:
                net.selftest_wait(limit_us)
            dt = time.perf_counter() - t0
            assert e.value.code == jet.JET_ETIMEOUT, e.value
            assert dt >= 2 * limit_us * 1e-6 and dt < 2 * limit_us * 1e-6 + 2.0, (limit_us, dt)
            after = net.contract(w.outputs)        # the same handle, right after the time-out
            assert np.array_equal(after, before)
        ref = np.array([oracle.amplitude(w.network.as_complex64(), x) for x in w.outputs])
        assert np.linalg.norm(after - ref) / np.linalg.norm(ref) <= 1e-5
    finally:
        net.close()
