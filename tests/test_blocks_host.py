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
