"""The launch graph of a small circuit (the n = 12 variational workload,
gate-by-gate path) captured once and replayed: the replay leaves exactly the
state a direct apply leaves (same kernels, same arguments), and both match the
oracle.  Complex128 (the workload's dtype) and complex64 (dense blocks fused to
4 and 5 qubits, tensor-core kernels inside the graph)."""
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


@pytest.mark.parametrize("dt,kw", [(torch.complex128, {}), (torch.complex128, {"fused": False}),
                                   (torch.complex64, {"blocks": 5})])
def test_replayed_graph_equals_direct_apply(qs, dt, kw):
    n = 12
    gates, params = W.variational(n, 10, "ladder", seed=0)
    circ = qs.Circuit(gates, n)
    direct = qs.State(n, dtype=dt)
    direct.reset()
    direct.apply_circuit(circ, params, **kw)
    want = direct.numpy()
    st = qs.State(n, dtype=dt)
    st.reset()
    cap = qs.CapturedCircuit(st, circ, params, **kw)
    for _ in range(3):
        st.reset()
        cap.replay()
        torch.cuda.synchronize()
        assert np.array_equal(st.numpy(), want)
    ref = oracle.apply_circuit(oracle.zero_state(n), n, gates, params)
    tol = 1e-12 if dt == torch.complex128 else 2e-5
    assert np.max(np.abs(want - ref)) < tol
    e = st.expect(qs.Observable(W.zz_chain(n)))[0]
    assert abs(e - oracle.expect(ref, n, W.zz_chain(n))) < (1e-12 if dt == torch.complex128 else 1e-5)
