"""Degenerate cases of the hot path against the FP64 oracle: one-qubit
registers (every gate kind, expectation, sampling, gradient), empty circuits
and observables, uneven batches holding one- and two-qubit registers, block
fusion wider than the register, and the tile engine at its smallest register
sizes (5..8 qubits: one pass, one or two thread bits) and below them (a clean
QS_EUNSUPPORTED when forced)."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"c64": torch.complex64, "c128": torch.complex128}
TOL = {"c64": 2e-5, "c128": 1e-12}


@pytest.fixture(scope="module")
def qs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10877_gb300 import qsim
    return qsim


def one_qubit_gates(seed):
    rs = np.random.default_rng(seed)
    return [W.Gate("H", (0,)), W.Gate("T", (0,)), W.Gate("RX", (0,), theta=0.3), W.Gate("S", (0,)),
            W.Gate("RZ", (0,), theta=-1.1), W.Gate("Y", (0,)), W.Gate("SHIFT", (0,), theta=0.7),
            W.Gate("RY", (0,), theta=2.2), W.Gate("MATRIX", (0,), matrix=W.haar_su2(seed)),
            W.Gate("X", (0,)), W.Gate("TDG", (0,)), W.Gate("PHASE", (0,), theta=0.4), W.Gate("Z", (0,)),
            W.Gate("SDG", (0,)), W.Gate("RX", (0,), theta=float(rs.uniform(-3, 3)))]


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_one_qubit_register(qs, dt):
    gates = one_qubit_gates(1)
    want = oracle.apply_circuit(oracle.zero_state(1), 1, gates)
    # gate by gate through instruct!, then as one circuit (fused single-qubit chain)
    st = qs.State(1, dtype=TDT[dt])
    st.reset()
    for g in gates:
        st.apply(g)
    assert np.max(np.abs(st.numpy() - want)) < TOL[dt]
    st2 = qs.State(1, dtype=TDT[dt])
    st2.reset()
    st2.apply_circuit(qs.Circuit(gates, 1))
    psi = st2.numpy()
    assert np.max(np.abs(psi - want)) < TOL[dt]
    for terms in ([(1.0, ((0, "Z"),))], [(0.5, ((0, "X"),)), (-2.0, ((0, "Y"),))]):
        got = st2.expect(qs.Observable(terms))[0]
        assert abs(got - oracle.expect(want, 1, terms)) < 10 * TOL[dt]
    u = W.shot_uniforms(256, seed=2)
    assert (st2.measure(u)[0] == oracle.sample(psi.astype(np.complex128), 1, u[0])).all()


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_one_qubit_gradient(qs, dt):
    gates = [W.Gate("RX", (0,), param=0), W.Gate("RZ", (0,), param=1), W.Gate("RY", (0,), param=2),
             W.Gate("SHIFT", (0,), param=1)]
    params = np.array([0.4, -1.3, 2.0])
    terms = [(1.0, ((0, "Z"),)), (0.3, ((0, "X"),))]
    circ = qs.Circuit(gates, 1)
    st = qs.State(1, dtype=TDT[dt])
    st.reset()
    st.apply_circuit(circ, params)
    loss, grad = qs.backward(st, circ, params, qs.Observable(terms))
    wl, wg = oracle.gradient(oracle.zero_state(1), 1, gates, params, terms)
    assert abs(loss - wl) < 10 * TOL[dt]
    assert np.max(np.abs(grad - wg)) < (1e-10 if dt == "c128" else 1e-4)


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_empty_circuit_and_observable(qs, dt):
    n = 4
    psi0 = W.haar_state(n, seed=3)
    circ = qs.Circuit([], n)
    for kw in ({}, {"fused": False}, {"blocks": 5}):
        st = qs.State(n, dtype=TDT[dt])
        st.upload(psi0)
        st.apply_circuit(circ, None, **kw)
        assert np.max(np.abs(st.numpy() - psi0)) < TOL[dt]
    assert st.expect(qs.Observable([]))[0] == 0.0
    terms = [(0.7, ((1, "Z"), (2, "Z"))), (0.2, ((3, "X"),))]
    loss, grad = qs.backward(st, circ, None, qs.Observable(terms))
    assert grad.shape == (0,)
    assert abs(loss - oracle.expect(psi0, n, terms)) < 10 * TOL[dt]


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_uneven_batch_with_one_and_two_qubit_registers(qs, dt):
    counts = [1, 3, 2, 1]
    inputs = [W.haar_state(k, seed=10 + r) for r, k in enumerate(counts)]
    gates = [W.Gate("H", (0,)), W.Gate("RX", (0,), theta=0.9), W.Gate("T", (0,)), W.Gate("X", (0,))]
    st = qs.State(counts, dtype=TDT[dt])
    st.upload(np.concatenate(inputs))
    for g in gates:
        st.apply(g)
    out = st.numpy()
    terms = [(1.0, ((0, "Z"),))]
    e = st.expect(qs.Observable(terms))
    off = 0
    for r, k in enumerate(counts):
        want = oracle.apply_circuit(inputs[r], k, gates)
        assert np.max(np.abs(out[off:off + (1 << k)] - want)) < TOL[dt], r
        assert abs(e[r] - oracle.expect(want, k, terms)) < 10 * TOL[dt], r
        off += 1 << k


@pytest.mark.parametrize("n", [1, 2, 3])
def test_blocks_wider_than_the_register(qs, n):
    gates = []
    rs = np.random.default_rng(n)
    for i in range(12):
        q = [int(x) for x in rs.permutation(n)]
        gates.append(W.Gate("MATRIX", (q[0],), matrix=W.haar_su2(i)))
        if n > 1:
            gates.append(W.cnot(q[0], q[1]))
    psi0 = W.haar_state(n, seed=4)
    st = qs.State(n, dtype=torch.complex128)
    st.upload(psi0)
    st.apply_circuit(qs.Circuit(gates, n), None, blocks=5)
    assert np.max(np.abs(st.numpy() - oracle.apply_circuit(psi0, n, gates))) < 1e-12


@pytest.mark.parametrize("n", [5, 6, 7, 8])
def test_tile_engine_smallest_registers(qs, n):
    for gates, params in ((W.qft(n, swaps=True), None), W.variational(n, 3, "ring", seed=n)):
        circ = qs.Circuit(gates, n, nparams=len(params) if params is not None else None)
        psi0 = W.haar_state(n, seed=n)
        st = qs.State(n, dtype=torch.complex64, nbatch=2)
        st.upload(np.concatenate([psi0, psi0]))
        st.apply_circuit(circ, params, tiles=True, tile_qubits=9)
        want = oracle.apply_circuit(psi0, n, gates, params)
        out = st.numpy().reshape(2, -1)
        assert np.max(np.abs(out - want[None, :])) < 2e-5


def test_tile_engine_rejects_registers_below_a_row(qs):
    from paper_1912_10877_gb300._native import QsimError
    n = 4
    st = qs.State(n, dtype=torch.complex64)
    st.reset()
    with pytest.raises(QsimError):
        st.apply_circuit(qs.Circuit(W.qft(n), n), None, tiles=True)
    # the default path still applies it
    st.apply_circuit(qs.Circuit(W.qft(n), n), None)
    assert np.max(np.abs(st.numpy() - oracle.apply_circuit(oracle.zero_state(n), n, W.qft(n)))) < 2e-5
