"""CPU checks of the k-qubit block fusion (host code, no device work): the
blocks the library fuses a circuit into, applied one by one as general
multi-qubit instructions by the oracle, reproduce the oracle's application of
the circuit itself (the matrix of a chain is the product of its parts,
Sec. "Matrix Representation"); every block respects the width limit unless it
is a single gate wider than the limit; and the planner only reorders gates
that share no qubit (checked through the same state equality on circuits
whose gates do not commute)."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def qs():
    from paper_1912_10877_gb300 import build as B
    B.build()
    from paper_1912_10877_gb300 import qsim
    return qsim


def mixed_circuit(n, seed):
    rs = np.random.default_rng(seed)
    gates = []
    for i in range(40):
        kind = i % 6
        perm = [int(x) for x in rs.permutation(n)]
        if kind == 0:
            gates.append(W.Gate("RX", (perm[0],), theta=float(rs.uniform(-3, 3))))
        elif kind == 1:
            gates.append(W.cnot(perm[0], perm[1]))
        elif kind == 2:
            gates.append(W.toffoli(perm[0], perm[1], perm[2]))
        elif kind == 3:
            gates.append(W.Gate("ROT", (perm[0], perm[1]), theta=float(rs.uniform(-3, 3)), paulis="XY"))
        elif kind == 4:
            gates.append(W.Gate("MATRIX", (perm[0],), matrix=W.haar_su2(seed * 100 + i)))
        else:
            gates.append(W.Gate("SWAP", (perm[0], perm[1]), (perm[2],), (0,)))
    return gates


def circuits():
    n = 8
    g, p = W.variational(n, 3, "ring", seed=1)
    yield "variational", n, g, p
    g, p = W.brickwork(n, 4, seed=2)
    yield "brickwork", n, g, p
    yield "qft", 7, W.qft(7, swaps=True), None
    yield "mixed", n, mixed_circuit(n, 3), None


@pytest.mark.parametrize("kmax", [1, 2, 3, 4, 5])
def test_blocks_reproduce_the_circuit(qs, kmax):
    for name, n, gates, params in circuits():
        circ = qs.Circuit(gates, n)
        blocks = qs.circuit_blocks(circ, params, kmax)
        psi = W.haar_state(n, seed=len(gates))
        want = oracle.apply_circuit(psi, n, gates, params)
        bgates = [W.Gate("MATRIX", q, matrix=m) for q, m in blocks]
        got = oracle.apply_circuit(psi, n, bgates)
        assert np.max(np.abs(got - want)) < 1e-12, (name, kmax)
        widest = max(len(set(g.locs) | set(g.ctrl_locs)) for g in gates)
        for q, m in blocks:
            assert len(q) <= max(kmax, widest)
            assert list(q) == sorted(q)
            # block matrices are unitary
            assert np.allclose(m.conj().T @ m, np.eye(len(m)), atol=1e-12)


def test_wider_blocks_mean_fewer_passes(qs):
    n = 10
    gates, params = W.brickwork(n, 6, seed=4)
    circ = qs.Circuit(gates, n)
    counts = [len(qs.circuit_blocks(circ, params, k, matrices=False)) for k in range(1, 6)]
    assert counts[0] <= len(gates)
    assert counts[-1] < counts[1] < counts[0], counts


def random_circuit(n, seed, ngates=60):
    """Random gates on random qubits, many of them overlapping, so that the
    planner's reordering (blocks moved past blocks of disjoint support, merged
    forward and backward) meets gates that do not commute."""
    rs = np.random.default_rng(seed)
    gates = []
    for _ in range(ngates):
        kind = int(rs.integers(0, 7))
        q = [int(x) for x in rs.permutation(n)]
        if kind == 0:
            gates.append(W.Gate("RY", (q[0],), theta=float(rs.uniform(-3, 3))))
        elif kind == 1:
            gates.append(W.cnot(q[0], q[1]))
        elif kind == 2:
            gates.append(W.Gate("H", (q[0],), (q[1],), (int(rs.integers(0, 2)),)))
        elif kind == 3:
            gates.append(W.Gate("MATRIX", (q[0], q[1]), matrix=_unitary(4, rs)))
        elif kind == 4:
            gates.append(W.Gate("SHIFT", (q[0],), (q[1], q[2]), (1, 0), theta=float(rs.uniform(-3, 3))))
        elif kind == 5:
            gates.append(W.Gate("MATRIX", (q[0], q[1], q[2]), matrix=_unitary(8, rs)))
        else:
            gates.append(W.Gate("SWAP", (q[0], q[1])))
    return gates


def _unitary(d, rs):
    a = rs.standard_normal((d, d)) + 1j * rs.standard_normal((d, d))
    q, r = np.linalg.qr(a)
    return q * (np.diag(r) / np.abs(np.diag(r)))


@pytest.mark.parametrize("seed", range(24))
def test_random_circuits_fused_in_any_width(qs, seed):
    n = 7
    gates = random_circuit(n, seed)
    circ = qs.Circuit(gates, n)
    psi = W.haar_state(n, seed=seed)
    want = oracle.apply_circuit(psi, n, gates)
    for kmax in (2, 3, 4, 5):
        blocks = qs.circuit_blocks(circ, None, kmax)
        got = oracle.apply_circuit(psi, n, [W.Gate("MATRIX", q, matrix=m) for q, m in blocks])
        assert np.max(np.abs(got - want)) < 1e-12, (seed, kmax)
        assert all(len(q) <= max(kmax, 3) for q, _ in blocks)
