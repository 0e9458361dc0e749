"""GPU parity of the reversible backward over k-qubit blocks (qs_backward_blocks)
against the oracle's reversible-adjoint gradient and loss: complex128 within
1e-10 relative (max-norm), complex64 within 2e-5 relative at n = 9 (measured
3.0e-6 with 5-qubit tensor-core blocks, 6.4e-7 without) and 3e-5 at n = 20
(FP32 states through the forward blocks and their adjoints on the tensor
cores; measured 7.2e-6), FP64 sums; block widths 1..5; controlled
rotations, shift and phase gates, multi-qubit Pauli rotations and a shared
parameter; the state is uncomputed to the circuit's input."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"c64": torch.complex64, "c128": torch.complex128}
GTOL = {"c64": 2e-5, "c128": 1e-10}


@pytest.fixture(scope="module")
def qs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10877_gb300 import qsim
    qsim.set_tensor_cores(1)
    return qsim


def rel(got, want):
    return float(np.max(np.abs(got - want)) / max(1e-300, np.max(np.abs(want))))


def param_circuit(n, seed):
    """Every parameterised kind the adjoint knows, controls included, one shared angle."""
    rs = np.random.default_rng(seed)
    gates, p = [], []

    def P():
        p.append(float(rs.uniform(0, 2 * np.pi)))
        return len(p) - 1

    for layer in range(3):
        for q in range(n):
            gates.append(W.Gate(["RX", "RY", "RZ"][(q + layer) % 3], (q,), param=P()))
        perm = [int(x) for x in rs.permutation(n)]
        gates.append(W.Gate("RX", (perm[0],), (perm[1],), (1,), param=P()))
        gates.append(W.Gate("SHIFT", (perm[2],), (perm[3],), (0,), param=P()))
        gates.append(W.Gate("PHASE", (perm[1],), param=P()))
        gates.append(W.Gate("ROT", (perm[0], perm[3]), param=P(), paulis="XY"))
        gates.append(W.cnot(perm[1], perm[2]))
        gates.append(W.Gate("MATRIX", (perm[3],), matrix=W.haar_su2(seed + layer)))
        gates.append(W.Gate("RZ", (perm[2],), param=0))  # shares parameter 0
    return gates, np.array(p)


def circuits(n):
    yield ("variational",) + W.variational(n, 3, "ring", seed=n)
    yield ("brickwork",) + W.brickwork(n, 4, seed=n)
    yield ("kinds",) + param_circuit(n, n)


@pytest.mark.parametrize("dt", ["c128", "c64"])
@pytest.mark.parametrize("kmax", [1, 3, 5])
def test_block_gradient_matches_oracle(qs, dt, kmax):
    n = 9
    terms = W.tfim(n, 1.0) if hasattr(W, "tfim") else W.zz_chain(n)
    for name, gates, params in circuits(n):
        circ = qs.Circuit(gates, n, nparams=len(params))
        obs = qs.Observable(terms)
        psi0 = W.haar_state(n, seed=3)
        st = qs.State(n, dtype=TDT[dt])
        st.upload(psi0)
        st.apply_circuit(circ, params, blocks=kmax)
        loss, grad = qs.backward_blocks(st, circ, params, obs, kmax=kmax)
        wl, wg = oracle.gradient(psi0, n, gates, params, terms)
        assert abs(loss - wl) < (1e-12 if dt == "c128" else 1e-5), (name, loss, wl)
        print(f"block gradient n=9 {dt} kmax={kmax} {name}: {rel(grad, wg):.2e}")
        assert rel(grad, wg) < GTOL[dt], (name, kmax, rel(grad, wg))
        # uncomputed back to the input
        back = st.numpy()
        assert np.max(np.abs(back - psi0)) < (1e-12 if dt == "c128" else 1e-4), name


def test_block_gradient_n20_against_fp64_adjoint(qs):
    # n = 20 complex64 through 5-qubit blocks (dense ones on the tensor cores) against
    # the per-gate FP64 adjoint of the library, itself pinned to the oracle
    n = 20
    gates, params = W.variational(n, 4, "ring", seed=20)
    circ = qs.Circuit(gates, n, nparams=len(params))
    obs = qs.Observable(W.zz_chain(n))
    st = qs.State(n, dtype=torch.complex64)
    st.reset()
    st.apply_circuit(circ, params, blocks=5)
    ref = qs.State(n, dtype=torch.complex128)
    ref.reset()
    ref.apply_circuit(circ, params)
    wl, wg = qs.backward(ref, circ, params, obs)
    loss, grad = qs.backward_blocks(st, circ, params, obs, kmax=5)
    print(f"block gradient n=20 vs FP64 adjoint: {rel(grad, wg):.2e}")
    assert abs(loss - wl) < 1e-5
    assert rel(grad, wg) < 3e-5, rel(grad, wg)  # measured on GB300: 7.2e-6


@pytest.mark.parametrize("kmax", [4, 5])
def test_block_gradient_tensor_core_gram_matches_cuda_core(qs, kmax):
    # 4- and 5-qubit supports: rho from the tensor-core Gram kernel (3xTF32, FP64 groups)
    # against the CUDA-core Gram kernel and the oracle
    n = 11
    for name, gates, params in circuits(n):
        circ = qs.Circuit(gates, n, nparams=len(params))
        terms = W.zz_chain(n) + [(0.4, ((3, "X"),))]
        obs = qs.Observable(terms)
        psi0 = W.haar_state(n, seed=5)
        out = {}
        for mode in (1, 0):
            qs.set_tensor_cores(mode)
            st = qs.State(n, dtype=torch.complex64)
            st.upload(psi0)
            st.apply_circuit(circ, params, blocks=kmax)
            out[mode] = qs.backward_blocks(st, circ, params, obs, kmax=kmax)
        qs.set_tensor_cores(1)
        wl, wg = oracle.gradient(psi0, n, gates, params, terms)
        for mode in (1, 0):
            assert abs(out[mode][0] - wl) < 1e-5
            assert rel(out[mode][1], wg) < 2e-5, (name, mode, rel(out[mode][1], wg))
        assert rel(out[1][1], out[0][1]) < 2e-5, name


def test_block_gradient_tensor_core_gram_many_groups(qs):
    # n = 24: 2^19 tuples per 5-qubit Gram, so every CTA of the TMA-fed Gram runs
    # several FP32 accumulation groups through both accumulator buffers; the
    # gradient with tensor cores on must match the CUDA-core Gram's
    n = 24
    gates, params = W.brickwork(n, 2, seed=7)
    circ = qs.Circuit(gates, n, nparams=len(params))
    obs = qs.Observable([(1.0, ((1, "Z"),)), (0.5, ((12, "X"), (13, "X")))])
    psi0 = W.haar_state(n, seed=8)
    out = {}
    for mode in (1, 0):
        qs.set_tensor_cores(mode)
        st = qs.State(n, dtype=torch.complex64)
        st.upload(psi0)
        st.apply_circuit(circ, params, blocks=5)
        out[mode] = qs.backward_blocks(st, circ, params, obs, kmax=5)
    qs.set_tensor_cores(1)
    print(f"block gradient n=24 tensor vs CUDA cores: {rel(out[1][1], out[0][1]):.2e}")
    assert abs(out[1][0] - out[0][0]) < 1e-5
    assert rel(out[1][1], out[0][1]) < 1.5e-5, rel(out[1][1], out[0][1])  # measured on GB300: 4.2e-6
