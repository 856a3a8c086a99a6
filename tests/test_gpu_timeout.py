"""Bounded device waits: the tensor-core exchange kernels bound every mbarrier wait; when a wait runs out
the kernel sets an error flag, waits for the copies and MMAs it has already issued, releases its tensor
memory and returns, and the host reports DF_E_TIMEOUT with the context still usable.

The test shortens the pipeline waits' budget to a few hundred cycles (DFHF_TC_WAIT_CYCLES, read by the
library at each launch), far below the latency of the first tensor-memory copy, so the waits run out in
every CTA; nothing faults and nothing hangs (the drains of work already issued keep their full budget).
The next call with the default budget gives the same K, bit for bit, as before.
"""
import os

import numpy as np
import pytest

from paper_1707_03771_gb300 import clusters

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1707_03771_gb300 import binding, build
    build.build()
    return binding


@pytest.mark.parametrize("slices", [3, 5])
def test_wait_runs_out_then_next_call_recovers(lib, slices):
    system = clusters.workload("water2")
    rng = np.random.default_rng(5)
    with lib.Handle(system) as h:
        h.build_B()
        C = np.linalg.qr(rng.normal(size=(h.n, h.nocc)))[0]
        D = 2 * C @ C.T
        J_ref, K_ref = h.jk(D, C, lib.DF_PREC_SPLIT, slices)
        os.environ["DFHF_TC_WAIT_CYCLES"] = "200"
        try:
            with pytest.raises(lib.DFError) as e:
                h.jk(D, C, lib.DF_PREC_SPLIT, slices)
        finally:
            del os.environ["DFHF_TC_WAIT_CYCLES"]
        assert e.value.code == lib.DF_E_TIMEOUT
        assert "timed out" in str(e.value)
        J, K = h.jk(D, C, lib.DF_PREC_SPLIT, slices)
        assert np.array_equal(K, K_ref)
        assert np.array_equal(J, J_ref)
        # the FP64 path on the same handle is unaffected
        _, K64 = h.jk(D, C)
        assert np.abs(K64 - K_ref).max() <= 2.0 ** (7 - 7 * slices) * np.abs(K64).max()
