"""The whole circuit of a small register in one cooperative launch
(qs_run_circuit_one_launch) against the oracle: the small workload (n = 12,
complex128, 10 layers of Rz Rx Rz + CNOT ladder) and its <sum Z_i Z_{i+1}>
evaluated in the same launch, at every block width and several grid sizes;
circuits with controls, multi-qubit gates and an even or odd number of
blocks (the result ends in either buffer); complex64; an empty circuit."""
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


@pytest.mark.parametrize("kmax", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("grid", [0, 16, 300])
def test_small_workload_one_launch(qs, kmax, grid):
    n = 12
    gates, params = W.variational(n, 10, "ladder", seed=0)
    terms = W.zz_chain(n)
    circ = qs.Circuit(gates, n)
    st = qs.State(n, dtype=torch.complex128)
    st.reset()
    out = qs.run_one_launch(st, circ, params, kmax=kmax, obs=qs.Observable(terms), grid_ctas=grid)
    st.sync()
    want = oracle.apply_circuit(oracle.zero_state(n), n, gates, params)
    assert np.max(np.abs(st.numpy() - want)) < 1e-12
    assert abs(float(out.item()) - oracle.expect(want, n, terms)) < 1e-12


@pytest.mark.parametrize("dt", ["c128", "c64"])
def test_mixed_gates_and_parities(qs, dt):
    n = 9
    rs = np.random.default_rng(4)
    base = [W.Gate("H", (0,)), W.toffoli(0, 3, 8), W.Gate("RY", (5,), (2,), (0,), theta=0.4),
            W.Gate("SWAP", (1, 7)), W.Gate("ROT", (2, 6), paulis="XZ", theta=1.3),
            W.Gate("MATRIX", (4, 0, 6), matrix=np.linalg.qr(rs.normal(size=(8, 8)) + 1j * rs.normal(size=(8, 8)))[0]),
            W.Gate("SHIFT", (8,), (1, 4), (1, 0), theta=2.2), W.Gate("T", (3,)), W.cnot(7, 2)]
    tol = 1e-12 if dt == "c128" else 2e-5
    for ng in (len(base), len(base) - 1, 1):
        gates = base[:ng]
        psi0 = W.haar_state(n, seed=ng)
        for kmax in (2, 3, 5):
            st = qs.State(n, dtype=torch.complex128 if dt == "c128" else torch.complex64)
            st.upload(psi0)
            qs.run_one_launch(st, qs.Circuit(gates, n), None, kmax=kmax)
            st.sync()
            want = oracle.apply_circuit(psi0.astype(np.complex64).astype(np.complex128) if dt == "c64" else psi0,
                                        n, gates)
            assert np.max(np.abs(st.numpy() - want)) < tol, (ng, kmax)


def test_empty_circuit_and_rejects(qs):
    n = 6
    psi0 = W.haar_state(n, seed=1)
    st = qs.State(n, dtype=torch.complex128)
    st.upload(psi0)
    out = qs.run_one_launch(st, qs.Circuit([], n), None, kmax=3, obs=qs.Observable(W.zz_chain(n)))
    st.sync()
    assert np.max(np.abs(st.numpy() - psi0)) < 1e-15
    assert abs(float(out.item()) - oracle.expect(psi0, n, W.zz_chain(n))) < 1e-12
    from paper_1912_10877_gb300 import QsimError
    with pytest.raises(QsimError):  # non-diagonal observable
        qs.run_one_launch(st, qs.Circuit([], n), None, kmax=3, obs=qs.Observable([(1.0, ((0, "X"),))]))
