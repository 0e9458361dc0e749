"""GPU parity of the k-qubit block path (QS_APPLY_BLOCKS) and the circuit
autotuner against the FP64 oracle: complex64 (tensor-core blocks where the
placement selects them) and complex128, k = 2..5, single registers and uneven
batches, up to n = 20.  Tolerances as elsewhere: 2e-5 (c64), 1e-12 (c128)."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"c64": 2e-5, "c128": 1e-12}
TDT = {"c64": torch.complex64, "c128": torch.complex128}


@pytest.fixture(scope="module")
def qs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10877_gb300 import qsim
    qsim.set_tensor_cores(1)
    return qsim


def mixed_circuit(n, seed):
    rs = np.random.default_rng(seed)
    gates = []
    for i in range(60):
        kind = i % 7
        perm = [int(x) for x in rs.permutation(n)]
        if kind == 0:
            gates.append(W.Gate("RX", (perm[0],), theta=float(rs.uniform(-3, 3))))
        elif kind == 1:
            gates.append(W.cnot(perm[0], perm[1]))
        elif kind == 2:
            gates.append(W.toffoli(perm[0], perm[1], perm[2]))
        elif kind == 3:
            gates.append(W.Gate("ROT", (perm[0], perm[1], perm[2]), theta=float(rs.uniform(-3, 3)), paulis="XYZ"))
        elif kind == 4:
            gates.append(W.Gate("MATRIX", (perm[0],), matrix=W.haar_su2(seed * 100 + i)))
        elif kind == 5:
            gates.append(W.Gate("H", (perm[0],)))
        else:
            gates.append(W.Gate("SWAP", (perm[0], perm[1]), (perm[2],), (1,)))
    return gates


def circuits(n):
    g, p = W.variational(n, 4, "ring", seed=n)
    yield "variational", g, p
    g, p = W.brickwork(n, 6, seed=n + 1)
    yield "brickwork", g, p
    yield "qft", W.qft(n, swaps=True), None
    yield "mixed", mixed_circuit(n, n), None


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_block_path_matches_oracle(qs, dt, k):
    n = 11
    for name, gates, params in circuits(n):
        circ = qs.Circuit(gates, n)
        psi = W.haar_state(n, seed=7)
        st = qs.State(n, dtype=TDT[dt])
        st.upload(psi)
        st.apply_circuit(circ, params, blocks=k)
        st.sync()
        want = oracle.apply_circuit(psi, n, gates, params)
        assert np.max(np.abs(st.numpy() - want)) < TOL[dt], (name, k)


def test_block_path_uneven_batch(qs):
    counts = [11, 8, 13, 9]
    n = 8
    gates, params = W.brickwork(n, 5, seed=3)
    circ = qs.Circuit(gates, n)
    st = qs.State(counts, dtype=torch.complex64)
    inputs = [W.haar_state(c, seed=c) for c in counts]
    st.upload(np.concatenate(inputs))
    st.apply_circuit(circ, params, blocks=5)
    st.sync()
    out = st.numpy()
    for r, c in enumerate(counts):
        seg = out[int(st.offsets[r]):int(st.offsets[r + 1])]
        assert np.max(np.abs(seg - oracle.apply_circuit(inputs[r], c, gates, params))) < TOL["c64"], r


def test_block_path_n20_tensor_cores(qs):
    # n = 20: 5-qubit blocks of a depth-10 variational ring circuit, the dense
    # ones on the tensor cores (forced), against the oracle element by element
    n = 20
    gates, params = W.variational(n, 10, "ring", seed=20)
    circ = qs.Circuit(gates, n)
    psi = W.haar_state(n, seed=20)
    want = oracle.apply_circuit(psi, n, gates, params)
    for mode in (2, 1):
        qs.set_tensor_cores(mode)
        st = qs.State(n, dtype=torch.complex64)
        st.upload(psi)
        st.apply_circuit(circ, params, blocks=5)
        st.sync()
        assert np.max(np.abs(st.numpy() - want)) < TOL["c64"], mode
    qs.set_tensor_cores(1)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_autotune_picks_a_valid_configuration(qs, dt):
    n = 16
    gates, params = W.variational(n, 4, "ladder", seed=16)
    circ = qs.Circuit(gates, n)
    st = qs.State(n, dtype=TDT[dt])
    st.reset()
    best, timings = qs.autotune(st, circ, params, reps=2)
    assert best in timings and timings[best] > 0
    assert all(v > 0 or v == -1 for v in timings.values())
    assert min(v for v in timings.values() if v > 0) == timings[best]
    if dt == "c64":
        assert any(f & 4 for f in timings)  # tile-engine candidates exist for complex64
    psi = W.haar_state(n, seed=3)
    st.upload(psi)
    st.apply_circuit(circ, params, flags=best)
    st.sync()
    want = oracle.apply_circuit(psi, n, gates, params)
    assert np.max(np.abs(st.numpy() - want)) < TOL[dt]
