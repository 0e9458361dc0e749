"""The tile engine's fused forward (complex64) against the FP64 oracle: circuits are
scheduled into passes over small tiles so that registers of 9..16 qubits span many
tiles and every pass / phase boundary is exercised.  Tolerance 2e-5 absolute."""
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


def check(qs, n, gates, params, tile, nbatch=1, seed=0):
    circ = qs.Circuit(gates, n, nparams=len(params) if params is not None else None)
    inputs = [W.haar_state(n, seed=seed + r) for r in range(nbatch)]
    st = qs.State(n, dtype=torch.complex64, nbatch=nbatch)
    st.upload(np.concatenate(inputs))
    st.apply_circuit(circ, params, tiles=True, tile_qubits=tile)
    out = st.numpy().reshape(nbatch, -1)
    for r in range(nbatch):
        want = oracle.apply_circuit(inputs[r], n, gates, params)
        err = np.max(np.abs(out[r] - want))
        assert err < 2e-5, (n, tile, r, err)


@pytest.mark.parametrize("n,tile", [(9, 9), (12, 9), (14, 10), (16, 13), (13, 13), (18, 11)])
def test_variational_ring(qs, n, tile):
    gates, params = W.variational(n, 3, "ring", seed=n)
    check(qs, n, gates, params, tile)


@pytest.mark.parametrize("n,tile", [(10, 9), (14, 10), (15, 13)])
def test_qft_with_swap_network(qs, n, tile):
    check(qs, n, W.qft(n, swaps=True), None, tile)


@pytest.mark.parametrize("n,tile", [(11, 9), (16, 12)])
def test_brickwork_matrices_and_cz(qs, n, tile):
    gates, params = W.brickwork(n, 4, seed=3)
    check(qs, n, gates, params, tile, nbatch=2)


def test_controls_inverse_controls_and_toffoli(qs):
    n = 14
    rs = np.random.default_rng(5)
    gates = []
    for i in range(120):
        perm = rs.permutation(n)
        nc = int(rs.integers(0, 4))
        name = ["X", "Y", "Z", "H", "T", "RX", "RY", "RZ", "SHIFT", "PHASE", "S"][i % 11]
        gates.append(W.Gate(name, (int(perm[0]),), tuple(int(x) for x in perm[1:1 + nc]),
                            tuple(int(x) for x in rs.integers(0, 2, nc)), theta=float(rs.uniform(-3, 3))))
        if i % 17 == 0:
            gates.append(W.Gate("SWAP", (int(perm[4]), int(perm[5])), (int(perm[6]),), (int(i % 2),)))
    check(qs, n, gates, None, 10)


def test_rejects_unsupported_when_forced(qs):
    from paper_1912_10877_gb300 import QsimError
    n = 12
    circ = qs.Circuit([W.Gate("ROT", (0, 5), theta=0.3, paulis="XY")], n)
    st = qs.State(n, dtype=torch.complex64)
    st.reset()
    with pytest.raises(QsimError):
        st.apply_circuit(circ, tiles=True, tile_qubits=9)
    st.apply_circuit(circ)  # the default path falls back to per-gate kernels


@pytest.mark.parametrize("n,tile,depth", [(10, 9, 3), (14, 10, 3), (16, 13, 2)])
def test_tiled_backward_vs_oracle(qs, n, tile, depth):
    gates, params = W.variational(n, depth, "ring", seed=n + 1)
    gates = gates + [W.Gate("RY", (3,), (1,), (0,), param=0), W.Gate("SHIFT", (2,), (5,), (1,), param=1),
                     W.Gate("PHASE", (n - 1,), (0,), (1,), param=2), W.Gate("H", (4,)),
                     W.Gate("MATRIX", (6,), matrix=W.haar_su2(3)), W.Gate("SWAP", (0, n - 1))]
    terms = W.tfim(n) + [(0.25, ((1, "Y"), (2, "X")))]
    circ = qs.Circuit(gates, n, nparams=len(params))
    st = qs.State(n, dtype=torch.complex64)
    st.reset()
    st.apply_circuit(circ, params, tiles=True, tile_qubits=tile)
    loss, grad = qs.backward_tiled(st, circ, params, qs.Observable(terms), tile_qubits=tile)
    rloss, rgrad = oracle.gradient(oracle.zero_state(n), n, gates, params, terms)
    assert abs(loss - rloss) < 1e-5
    assert np.max(np.abs(grad - rgrad)) / np.max(np.abs(rgrad)) < 1e-4


@pytest.mark.parametrize("n,tile,seed", [(13, 9, 0), (13, 10, 1), (16, 13, 2)])
def test_runs_of_diagonal_gates(qs, n, tile, seed):
    """Long runs of diagonal gates between a few Hadamards: phase gates with
    thread-bit controls, single phase-local controls of either value, general
    (non-unitary, one with a zero entry) diagonal matrices, all folded into
    per-bit factors that the non-diagonal gates settle first."""
    rs = np.random.default_rng(seed)
    gates = []
    for i in range(300):
        perm = [int(x) for x in rs.permutation(n)]
        if i % 23 == 0:
            gates.append(W.Gate("H", (perm[0],)))
            continue
        nc = int(rs.integers(0, 3))
        ctrls, vals = tuple(perm[1:1 + nc]), tuple(int(v) for v in rs.integers(0, 2, nc))
        kind = i % 5
        if kind == 0:
            gates.append(W.Gate("SHIFT", (perm[0],), ctrls, vals, theta=float(rs.uniform(-3, 3))))
        elif kind == 1:
            gates.append(W.Gate("RZ", (perm[0],), ctrls, vals, theta=float(rs.uniform(-3, 3))))
        elif kind == 2:
            d = rs.uniform(0.8, 1.25, 2) * np.exp(1j * rs.uniform(-3, 3, 2))
            if i % 47 == 2:
                d[int(i % 2)] = 0.0
            gates.append(W.Gate("MATRIX", (perm[0],), ctrls, vals, matrix=np.diag(d)))
        elif kind == 3:
            gates.append(W.Gate(["T", "S", "Z"][i % 3], (perm[0],), ctrls, vals))
        else:
            gates.append(W.Gate("RX", (perm[0],), ctrls, vals, theta=float(rs.uniform(-3, 3))))
    circ = qs.Circuit(gates, n)
    psi = W.haar_state(n, seed=seed)
    st = qs.State(n, dtype=torch.complex64)
    st.upload(psi)
    st.apply_circuit(circ, None, tiles=True, tile_qubits=tile)
    got = st.numpy()
    want = oracle.apply_circuit(psi, n, gates)
    scale = max(1.0, float(np.max(np.abs(want))))
    assert np.max(np.abs(got - want)) < 2e-5 * scale
