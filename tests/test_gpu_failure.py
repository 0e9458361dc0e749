"""Failure detection without a GPU fault: a device wait that nothing satisfies
runs through the bounded mbarrier wait of the tensor-core kernels, gives up
after its limit, and the host reads QS_ETIMEDOUT through the device status
word; the context stays usable (a gate runs correctly afterwards)."""
import ctypes
import time

import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10877_gb300 import qsim
    return qsim


def test_bounded_wait_reports_timeout_and_context_survives(qs):
    from paper_1912_10877_gb300 import _native as N
    res = (ctypes.c_int * 3)()
    t0 = time.perf_counter()
    rc = N.lib().qs_selftest_bounded_wait(20.0, res)
    dt = time.perf_counter() - t0
    assert rc == N.QS_ETIMEDOUT, N.lib().qs_last_error()
    assert res[0] == 0 and res[1] == 1
    assert 15_000 <= res[2] < 1_000_000, res[2]  # waited about its 20 ms limit
    assert dt < 10.0
    # the status word was cleared and the device still computes
    n = 8
    psi = W.haar_state(n, seed=1)
    st = qs.State(n, dtype=torch.complex64)
    st.upload(psi)
    g = W.Gate("H", (3,))
    st.apply(g)
    st.sync()
    assert np.max(np.abs(st.numpy() - oracle.apply_circuit(psi, n, [g]))) < 2e-5
