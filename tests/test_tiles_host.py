"""CPU checks of the tile engine's scheduler (host code, no device work): the
order in which the engine applies a circuit's gates (SWAPs rewritten as three
controlled X gates), applied gate by gate by the oracle, reproduces the
oracle's application of the circuit itself; passes never decrease along the
order, every gate appears exactly once, and wider tiles never need more passes.
Reordering is only valid between gates on disjoint qubits (Sec. "Representing
Quantum Circuits": a chain is the product of its parts in order), so random
circuits with overlapping controls, diagonal runs and swaps probe it."""
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


def expanded(gates):
    """The engine's SWAP rewrite: X(b) ctrl a, X(a) ctrl b, X(b) ctrl a, plus the SWAP's controls."""
    out = []
    for g in gates:
        if g.name != "SWAP":
            out.append(g)
            continue
        a, b = g.locs
        for t, c in ((b, a), (a, b), (b, a)):
            out.append(W.Gate("X", (t,), tuple(g.ctrl_locs) + (c,), tuple(g.ctrl_vals) + (1,)))
    return out


def random_circuit(n, seed, ngates=150):
    rs = np.random.default_rng(seed)
    names = ["H", "X", "Y", "Z", "T", "S", "RX", "RY", "RZ", "SHIFT", "PHASE", "SDG", "TDG"]
    gates = []
    for i in range(ngates):
        q = [int(x) for x in rs.permutation(n)]
        if i % 19 == 7:
            nc = int(rs.integers(0, 2))
            gates.append(W.Gate("SWAP", (q[0], q[1]), tuple(q[2:2 + nc]), tuple(int(v) for v in rs.integers(0, 2, nc))))
            continue
        nc = int(rs.integers(0, 4))
        name = names[int(rs.integers(0, len(names)))]
        if i % 11 == 3:
            gates.append(W.Gate("MATRIX", (q[0],), tuple(q[1:1 + nc]), tuple(int(v) for v in rs.integers(0, 2, nc)),
                                matrix=W.haar_su2(seed * 1000 + i)))
            continue
        gates.append(W.Gate(name, (q[0],), tuple(q[1:1 + nc]), tuple(int(v) for v in rs.integers(0, 2, nc)),
                            theta=float(rs.uniform(-3, 3))))
    return gates


def check_schedule(qs, n, gates, params, tile):
    circ = qs.Circuit(gates, n, nparams=len(params) if params is not None else None)
    order, passes = qs.tile_order(circ, tile)
    ex = expanded(gates)
    assert sorted(order.tolist()) == list(range(len(ex)))
    assert np.all(np.diff(passes) >= 0)
    psi = W.haar_state(n, seed=n + tile)
    want = oracle.apply_circuit(psi, n, gates, params)
    got = oracle.apply_circuit(psi, n, [ex[i] for i in order], params)
    assert np.max(np.abs(got - want)) < 1e-12, (n, tile)
    return int(passes[-1]) + 1 if len(passes) else 0


@pytest.mark.parametrize("seed", range(32))
def test_random_circuits_keep_their_result(qs, seed):
    n = [9, 10, 11, 12][seed % 4]
    gates = random_circuit(n, seed)
    npass = {tile: check_schedule(qs, n, gates, None, tile) for tile in (9, 10, 11, 13)}
    assert npass[13] <= npass[11] <= npass[10] <= npass[9], npass


@pytest.mark.parametrize("n", [5, 8, 14, 16])
def test_workload_circuits_keep_their_result(qs, n):
    for gates, params in ((W.qft(n, swaps=True), None), W.variational(n, 3, "ring", seed=n),
                          W.brickwork(n, 4, seed=n)):
        for tile in (9, 13):
            check_schedule(qs, n, gates, params, tile)


def test_unsupported_circuits_are_refused(qs):
    from paper_1912_10877_gb300._native import QsimError
    with pytest.raises(QsimError):
        qs.tile_order(qs.Circuit(W.qft(4), 4))
    with pytest.raises(QsimError):
        qs.tile_order(qs.Circuit([W.Gate("ROT", (0, 3), theta=0.2, paulis="XX")], 8))


def test_many_controls_schedule(qs):
    # controls are predicates on the amplitude index, so gates with many controls
    # (here up to 6) schedule like any other single-target gate
    n = 12
    rs = np.random.default_rng(3)
    gates = []
    for i in range(120):
        q = [int(x) for x in rs.permutation(n)]
        nc = int(rs.integers(0, 7))
        name = ["H", "X", "RY", "T", "SHIFT", "Z"][i % 6]
        gates.append(W.Gate(name, (q[0],), tuple(q[1:1 + nc]), tuple(int(v) for v in rs.integers(0, 2, nc)),
                            theta=float(rs.uniform(-3, 3))))
    for tile in (9, 13):
        check_schedule(qs, n, gates, None, tile)
