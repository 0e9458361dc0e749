"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by
element, on the same seeded inputs.  Tolerances (absolute, states normalised to
1): complex128 1e-12, complex64 2e-5 on amplitudes; expectations 1e-12 (c128)
and 1e-5 (c64, FP64 reduction of FP32 amplitudes); sample indices bit-exact."""
import math

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
    return qsim


def run_gpu(qs, psi, n, gates, params=None, dt="c128", nbatch=1):
    st = qs.State(n, dtype=TDT[dt], nbatch=nbatch)
    st.upload(np.tile(psi, nbatch))
    for g in gates:
        st.apply(g, params)
    return st.numpy().reshape(nbatch, -1)


def rand_unitary(k, rs):
    d = 1 << k
    a = rs.standard_normal((d, d)) + 1j * rs.standard_normal((d, d))
    q, r = np.linalg.qr(a)
    return q * (np.diag(r) / np.abs(np.diag(r)))


NAMED = ["X", "Y", "Z", "H", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "SHIFT", "PHASE"]


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 2, 5, 11])
def test_named_single_qubit_gates_every_loc(qs, dt, n):
    rs = np.random.default_rng(n)
    psi = W.haar_state(n, seed=100 + n)
    for name in NAMED:
        for t in range(n):
            g = W.Gate(name, (t,), theta=float(rs.uniform(-4, 4)))
            got = run_gpu(qs, psi, n, [g], dt=dt)[0]
            want = oracle.apply_circuit(psi, n, [g])
            assert np.max(np.abs(got - want)) < TOL[dt], (name, t)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_controlled_gates_all_placements(qs, dt):
    n = 6
    rs = np.random.default_rng(3)
    psi = W.haar_state(n, seed=7)
    for trial in range(80):
        name = NAMED[trial % len(NAMED)]
        perm = rs.permutation(n)
        nc = 1 + trial % 3
        t, cl = int(perm[0]), tuple(int(x) for x in perm[1:1 + nc])
        if trial % 5 == 0:
            cl = (0,) + tuple(c for c in cl if c != 0)[: nc - 1] if t != 0 else cl  # control on bit 0
        cv = tuple(int(x) for x in rs.integers(0, 2, len(cl)))
        g = W.Gate(name, (t,), cl, cv, theta=float(rs.uniform(-4, 4)))
        got = run_gpu(qs, psi, n, [g], dt=dt)[0]
        want = oracle.apply_circuit(psi, n, [g])
        assert np.max(np.abs(got - want)) < TOL[dt], (name, t, cl, cv)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_multi_qubit_matrices_swap_rot(qs, dt):
    rs = np.random.default_rng(11)
    for trial in range(40):
        n = int(rs.integers(3, 10))
        k = int(rs.integers(1, min(n, 5) + 1))
        nc = int(rs.integers(0, min(n - k, 2) + 1))
        perm = rs.permutation(n)
        locs = tuple(int(x) for x in perm[:k])
        cl = tuple(int(x) for x in perm[k:k + nc])
        cv = tuple(int(x) for x in rs.integers(0, 2, nc))
        kind = trial % 4
        if kind == 0:
            U = rand_unitary(k, rs)
        elif kind == 1:  # diagonal
            U = np.diag(np.exp(1j * rs.uniform(-3, 3, 1 << k)))
        else:  # permutation with phases
            P = np.eye(1 << k)[rs.permutation(1 << k)]
            U = P * np.exp(1j * rs.uniform(-3, 3, 1 << k))[:, None]
        psi = W.haar_state(n, seed=trial)
        g = W.Gate("MATRIX", locs, cl, cv, matrix=U)
        got = run_gpu(qs, psi, n, [g], dt=dt)[0]
        want = oracle.apply_circuit(psi, n, [g])
        assert np.max(np.abs(got - want)) < TOL[dt], (n, k, locs, cl, kind)
    n = 7
    psi = W.haar_state(n, seed=1)
    gates = [W.Gate("SWAP", (0, 6)), W.Gate("SWAP", (3, 2), (5,), (0,)),
             W.Gate("ROT", (1, 4), theta=0.3, paulis="XY"), W.Gate("ROT", (0, 2, 5), theta=-1.1, paulis="ZXY"),
             W.toffoli(0, 1, 6), W.Gate("Z", (6,), (0, 3), (1, 0))]
    got = run_gpu(qs, psi, n, gates, dt=dt)[0]
    assert np.max(np.abs(got - oracle.apply_circuit(psi, n, gates))) < TOL[dt]


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_uniform_and_uneven_batches(qs, dt):
    n = 8
    gates, params = W.variational(n, 2, "ring", seed=5)
    psi = W.haar_state(n, seed=2)
    got = run_gpu(qs, psi, n, gates, params, dt=dt, nbatch=3)
    want = oracle.apply_circuit(psi, n, gates, params)
    for r in range(3):
        assert np.max(np.abs(got[r] - want)) < TOL[dt]
    counts = [3, 7, 5, 9]
    st = qs.State(counts, dtype=TDT[dt])
    inputs = [W.haar_state(c, seed=c) for c in counts]
    st.upload(np.concatenate(inputs))
    g = [W.Gate("H", (1,)), W.cnot(0, 2), W.Gate("RY", (2,), (1,), (0,), theta=0.4)]
    for x in g:
        st.apply(x)
    out = st.numpy()
    for r, c in enumerate(counts):
        seg = out[int(st.offsets[r]):int(st.offsets[r + 1])]
        assert np.max(np.abs(seg - oracle.apply_circuit(inputs[r], c, g))) < TOL[dt]


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_circuit_object_small_variational(qs, dt):
    # n = 12, 10 layers of Rz Rx Rz + CNOT ladder from |0>, <sum Z_i Z_{i+1}> (open)
    n = 12
    terms = W.zz_chain(n)
    for seed in range(3):
        gates, params = W.variational(n, 10, "ladder", seed=seed)
        circ = qs.Circuit(gates, n)
        st = qs.State(n, dtype=TDT[dt])
        st.reset()
        st.apply_circuit(circ, params)
        want = oracle.apply_circuit(oracle.zero_state(n), n, gates, params)
        assert np.max(np.abs(st.numpy() - want)) < TOL[dt]
        e = st.expect(qs.Observable(terms))[0]
        assert abs(e - oracle.expect(want, n, terms)) < (1e-12 if dt == "c128" else 1e-5)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_qft_with_swaps_on_basis_state(qs, dt):
    n = 10
    x = W.random_basis(n, seed=3)
    circ = qs.Circuit(W.qft(n, swaps=True), n)
    st = qs.State(n, dtype=TDT[dt])
    st.reset([x])
    st.apply_circuit(circ)
    want = oracle.apply_circuit(oracle.basis_state(n, x), n, W.qft(n, swaps=True))
    assert np.max(np.abs(st.numpy() - want)) < TOL[dt]


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_expectation_random_pauli_sums(qs, dt):
    rs = np.random.default_rng(9)
    for n in (1, 4, 10):
        psi = W.haar_state(n, seed=n)
        terms = []
        for _ in range(20):
            q = rs.permutation(n)[: rs.integers(1, n + 1)]
            terms.append((float(rs.standard_normal()), tuple((int(l), "XYZ"[rs.integers(3)]) for l in q)))
        st = qs.State(n, dtype=TDT[dt], nbatch=2)
        st.upload(np.tile(psi, 2))
        e = st.expect(qs.Observable(terms))
        want = oracle.expect(psi.astype(np.complex64).astype(np.complex128) if dt == "c64" else psi, n, terms)
        assert np.max(np.abs(e - want)) < (1e-12 if dt == "c128" else 1e-9)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n", [3, 10, 21])
def test_sampling_bit_exact(qs, dt, n):
    psi = W.haar_state(n, seed=n + 50)
    st = qs.State(n, dtype=TDT[dt])
    st.upload(psi)
    u = W.shot_uniforms(4096 if n < 21 else 512, seed=n)
    got = st.measure(u)[0]
    # both sides sample the same stored state (complex64 promoted exactly)
    want = oracle.sample(st.numpy().astype(np.complex128), n, u[0])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_seeded_sampling_bit_exact(qs, dt):
    # the seed alone fixes the indices: device SplitMix64 uniforms against the oracle's
    counts = [3, 10, 21, 7]
    st = qs.State(counts, dtype=TDT[dt])
    st.upload(np.concatenate([W.haar_state(c, seed=c + 60) for c in counts]))
    nshots = 700
    for seed in (0, 2 ** 63 + 12345):
        got = st.measure_seeded(seed, nshots)
        out = st.numpy()
        for r, c in enumerate(counts):
            seg = out[int(st.offsets[r]):int(st.offsets[r + 1])].astype(np.complex128)
            assert np.array_equal(got[r], oracle.sample_seeded(seg, c, seed, nshots, reg=r)), (dt, seed, r)
    # collapse from a seed on one register
    n = 6
    psi = W.haar_state(n, seed=5)
    s1 = qs.State(n, dtype=TDT[dt])
    s1.upload(psi)
    x = int(s1.measure_seeded(99, 1, collapse=True)[0, 0])
    stored = psi.astype(np.complex64).astype(np.complex128) if dt == "c64" else psi
    assert x == int(oracle.sample_seeded(stored, n, 99, 1)[0])


def test_measure_listing_and_collapse(qs):
    st = qs.State(4, dtype=torch.complex128)
    st.reset()
    st.apply(W.Gate("X", (1,)))
    assert list(st.measure(W.shot_uniforms(3, seed=0))[0]) == [2, 2, 2]
    n = 6
    psi = W.haar_state(n, seed=4)
    st = qs.State(n, dtype=torch.complex128)
    st.upload(psi)
    u = np.array([[0.37]])
    x = int(st.measure(u, collapse=True)[0, 0])
    assert x == int(oracle.sample(psi, n, u[0])[0])
    assert np.max(np.abs(st.numpy() - oracle.collapse(psi, n, x))) < 1e-15


def test_batched_measure_uneven(qs):
    counts = [2, 9, 5]
    st = qs.State(counts, dtype=torch.complex64)
    inputs = [W.haar_state(c, seed=c + 3) for c in counts]
    st.upload(np.concatenate(inputs))
    u = W.shot_uniforms(300, seed=8, nreg=3)
    got = st.measure(u)
    out = st.numpy()
    for r, c in enumerate(counts):
        seg = out[int(st.offsets[r]):int(st.offsets[r + 1])].astype(np.complex128)
        assert np.array_equal(got[r], oracle.sample(seg, c, u[r]))


# ---------------------------------------------------------------- gradients

def test_symad_golden_on_gpu(qs):
    from conftest import read_golden
    g = read_golden("symad.txt")
    gates, params = W.symad_circuit()
    circ = qs.Circuit(gates, 3)
    obs = qs.Observable(W.heisenberg(3))
    st = qs.State(3, dtype=torch.complex128)
    st.reset()
    st.apply_circuit(circ, params)
    loss, grad = qs.backward(st, circ, params, obs)
    assert abs(loss - g["energy"]) < 1e-14
    assert np.allclose(grad, [g["grad_alpha"], g["grad_beta"], g["grad_gamma"]], rtol=1e-13, atol=0)


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_adjoint_vs_oracle_and_checkpoints(qs, dt):
    n = 9
    gates, params = W.variational(n, 4, "ring", seed=6)
    gates = gates + [W.Gate("SHIFT", (2,), (5,), (1,), param=len(params)),
                     W.Gate("ROT", (0, 7), param=len(params) + 1, paulis="YX"),
                     W.Gate("PHASE", (4,), (8,), (0,), param=0)]
    params = np.append(params, [0.3, -0.8])
    terms = W.tfim(n)
    circ = qs.Circuit(gates, n)
    obs = qs.Observable(terms)
    rloss, rgrad = oracle.gradient(oracle.zero_state(n), n, gates, params, terms)
    scale = np.max(np.abs(rgrad))
    tol = 1e-10 if dt == "c128" else 2e-5
    for every in (0, 7, 40):
        st = qs.State(n, dtype=TDT[dt])
        st.reset()
        ck = qs.checkpoint_buffer(st, circ, every) if every else None
        qs.apply_circuit_ckpt(st, circ, params, every, ck)
        loss, grad = qs.backward(st, circ, params, obs, every, ck)
        assert abs(loss - rloss) < (1e-12 if dt == "c128" else 1e-5)
        assert np.max(np.abs(grad - rgrad)) / scale < tol, every


def test_adjoint_matches_finite_differences_on_gpu(qs):
    n = 6
    gates, params = W.variational(n, 3, "ladder", seed=2)
    terms = W.tfim(n)
    circ = qs.Circuit(gates, n)
    obs = qs.Observable(terms)
    st = qs.State(n, dtype=torch.complex128)
    st.reset()
    st.apply_circuit(circ, params)
    _, grad = qs.backward(st, circ, params, obs)
    fd = oracle.fd_gradient(oracle.zero_state(n), n, gates, params, terms, h=1e-5, which=range(0, len(params), 5))
    for i, v in fd.items():
        assert abs(grad[i] - v) < 1e-8


def test_autograd_function(qs):
    from paper_1912_10877_gb300.autograd import expectation
    n = 5
    gates, params = W.variational(n, 2, "ladder", seed=1)
    circ = qs.Circuit(gates, n)
    obs = qs.Observable(W.tfim(n))
    p = torch.tensor(params, dtype=torch.float64, requires_grad=True)
    loss = expectation(p, circ, obs, torch.complex128)
    loss.backward()
    rloss, rgrad = oracle.gradient(oracle.zero_state(n), n, gates, params, W.tfim(n))
    assert abs(loss.item() - rloss) < 1e-12
    assert np.allclose(p.grad.numpy(), rgrad, atol=1e-11)


def test_errors_are_reported(qs):
    st = qs.State(3, dtype=torch.complex64)
    st.reset()
    from paper_1912_10877_gb300 import QsimError
    with pytest.raises(QsimError):
        st.apply(W.Gate("X", (3,)))
    with pytest.raises(QsimError):
        st.apply(W.Gate("X", (1,), (1,)))
    with pytest.raises(QsimError):
        st.measure(np.array([[1.5]]))
