"""Pins for the FP64 oracle: each test checks it against something other than itself
(values the paper prints, closed forms, library routines, brute force, invariants)."""
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import oracle
import workloads as W
from conftest import read_golden

PAULI = {
    "I": np.eye(2, dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
}


def rand_unitary(k, rs):
    d = 1 << k
    a = rs.standard_normal((d, d)) + 1j * rs.standard_normal((d, d))
    q, r = np.linalg.qr(a)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def tensor_apply(psi, n, U, locs, ctrl_locs=(), ctrl_vals=()):
    """Independent route: reshape the state to a rank-n tensor (axis a <-> qubit n-1-a) and
    contract the gate tensor on the target axes with einsum; controls select a slice."""
    k = len(locs)
    T = psi.reshape((2,) * n)
    Ut = U.reshape((2,) * (2 * k))  # axes: out bits (k-1..0), in bits (k-1..0)
    letters = "abcdefghijklmnopqrstuvwxyz"
    st = list(letters[:n])
    outs = list("ABCDEFGHIJ"[:k])
    ins = [st[n - 1 - locs[j]] for j in reversed(range(k))]  # in-bit order k-1..0
    res = list(st)
    for pos, j in enumerate(reversed(range(k))):
        res[n - 1 - locs[j]] = outs[pos]
    expr = "".join(outs) + "".join(ins) + "," + "".join(st) + "->" + "".join(res)
    new = np.einsum(expr, Ut, T)
    if ctrl_locs:
        sl = [slice(None)] * n
        for c, v in zip(ctrl_locs, ctrl_vals):
            sl[n - 1 - c] = v
        out = T.copy()
        out[tuple(sl)] = new[tuple(sl)]
        new = out
    return new.reshape(-1)


def kron_full(n, ops):
    """Textbook dense operator: kron over qubits n-1 .. 0 of the 2x2 matrix on each qubit."""
    M = np.eye(1, dtype=complex)
    for q in reversed(range(n)):
        M = np.kron(M, ops.get(q, PAULI["I"]))
    return M


def full_matrix(n, gates, params=None):
    """Columns = the oracle applied to each basis vector."""
    dim = 1 << n
    return np.stack([oracle.apply_circuit(oracle.basis_state(n, x), n, gates, params)
                     for x in range(dim)], axis=1)


# ------------------------------------------------------------------ conventions

def test_instruct_measure_listing():
    g = read_golden("instruct_measure.txt")
    n = int(g["n"])
    psi = oracle.apply_circuit(oracle.zero_state(n), n, [W.Gate("X", (int(g["x_qubit_paper"]) - 1,))])
    shots = oracle.sample(psi, n, W.shot_uniforms(int(g["shots"]), seed=3)[0])
    assert list(shots) == [int(g["expected_index"])] * int(g["shots"])


def test_shift_listing_matrices():
    th = 0.37
    # shift(theta) |> mat == diag(1, e^{i theta})
    M1 = full_matrix(1, [W.Gate("SHIFT", (0,), theta=th)])
    assert np.allclose(M1, np.diag([1, np.exp(1j * th)]), atol=1e-15)
    # control(2, 1, 2=>shift(theta)) |> mat == diag(1, 1, 1, e^{i theta})
    M2 = full_matrix(2, [W.Gate("SHIFT", (1,), (0,), (1,), theta=th)])
    assert np.allclose(M2, np.diag([1, 1, 1, np.exp(1j * th)]), atol=1e-15)


def test_single_qubit_gates_match_kron_formula():
    rs = np.random.default_rng(1)
    n = 5
    names = ["X", "Y", "Z", "H", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "SHIFT", "PHASE"]
    for name in names:
        for t in range(n):
            th = rs.uniform(-3, 3)
            g = W.Gate(name, (t,), theta=th)
            U = oracle.gate_matrix(g, th)
            full = kron_full(n, {t: U})
            psi = W.haar_state(n, seed=t + 17)
            assert np.allclose(oracle.apply_circuit(psi, n, [g]), full @ psi, atol=1e-13)


def test_named_gates_are_their_textbook_matrices():
    # App. "Builtin Block Types": the constant gates written out here, not taken
    # from the oracle; the oracle applied to basis vectors must reproduce them
    # entry by entry (a global sign or phase counts as a mistake here: controlled
    # versions expose it)
    r2 = 1 / np.sqrt(2)
    th = 0.61
    want = {
        "X": PAULI["X"], "Y": PAULI["Y"], "Z": PAULI["Z"],
        "H": np.array([[r2, r2], [r2, -r2]]),
        "S": np.diag([1, 1j]), "SDG": np.diag([1, -1j]),
        "T": np.diag([1, (1 + 1j) * r2]), "TDG": np.diag([1, (1 - 1j) * r2]),
        "SHIFT": np.diag([1, np.exp(1j * th)]), "PHASE": np.exp(1j * th) * np.eye(2),
    }
    for name, U in want.items():
        g = W.Gate(name, (0,), theta=th)
        assert np.allclose(full_matrix(1, [g]), U, atol=1e-15), name
        gc = W.Gate(name, (1,), (0,), (1,), theta=th)
        P0, P1 = np.diag([1, 0]), np.diag([0, 1])
        assert np.allclose(full_matrix(2, [gc]), np.kron(np.eye(2), P0) + np.kron(U, P1), atol=1e-15), name


def test_cnot_matches_projector_kron():
    n = 4
    P0 = np.diag([1, 0]).astype(complex)
    P1 = np.diag([0, 1]).astype(complex)
    for c in range(n):
        for t in range(n):
            if c == t:
                continue
            full = kron_full(n, {c: P0}) + kron_full(n, {c: P1, t: PAULI["X"]})
            psi = W.haar_state(n, seed=10 * c + t)
            assert np.allclose(oracle.apply_circuit(psi, n, [W.cnot(c, t)]), full @ psi, atol=1e-14)


def test_random_multiqubit_controlled_gates_vs_tensor_contraction():
    rs = np.random.default_rng(7)
    for trial in range(60):
        n = int(rs.integers(2, 8))
        k = int(rs.integers(1, min(n, 5) + 1))
        nc = int(rs.integers(0, min(n - k, 3) + 1))
        perm = rs.permutation(n)
        locs = tuple(int(x) for x in perm[:k])
        cl = tuple(int(x) for x in perm[k:k + nc])
        cv = tuple(int(x) for x in rs.integers(0, 2, nc))
        U = rand_unitary(k, rs)
        psi = W.haar_state(n, seed=trial)
        got = oracle.apply_circuit(psi, n, [W.Gate("MATRIX", locs, cl, cv, matrix=U)])
        want = tensor_apply(psi, n, U, locs, cl, cv)
        assert np.allclose(got, want, atol=1e-13), (n, k, locs, cl, cv)


def test_rotations_are_matrix_exponentials():
    rs = np.random.default_rng(3)
    for name, P in (("RX", "X"), ("RY", "Y"), ("RZ", "Z")):
        th = rs.uniform(-7, 7)
        U = oracle.gate_matrix(W.Gate(name, (0,), theta=th), th)
        assert np.allclose(U, scipy.linalg.expm(-0.5j * th * PAULI[P]), atol=1e-14)
    for paulis in ("XX", "XY", "ZY", "XYZ"):
        th = rs.uniform(-7, 7)
        k = len(paulis)
        U = oracle.gate_matrix(W.Gate("ROT", tuple(range(k)), theta=th, paulis=paulis), th)
        S = np.eye(1, dtype=complex)
        for p in reversed(paulis):  # bit j <-> target j: kron(sigma_{k-1}, ..., sigma_0)
            S = np.kron(S, PAULI[p])
        assert np.allclose(U, scipy.linalg.expm(-0.5j * th * S), atol=1e-13)
    # shift(theta) = e^{i theta / 2} Rz(theta)
    th = 1.234
    assert np.allclose(oracle.gate_matrix(W.Gate("SHIFT", (0,), theta=th), th),
                       np.exp(0.5j * th) * scipy.linalg.expm(-0.5j * th * PAULI["Z"]), atol=1e-14)


def test_iswap_permmatrix_printout():
    # App. "Matrix Types": PermMatrix([1,3,2,4], [1, i, i, 1]) prints rows
    # [1 0 0 0; 0 0 i 0; 0 i 0 0; 0 0 0 1]; as a gate on (l0, l1) it maps |01> <-> |10> with i.
    want = np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]])
    # ISWAP = exp(i pi/4 (XX + YY)) (library expm of the Pauli sum)
    XX = np.kron(PAULI["X"], PAULI["X"])
    YY = np.kron(PAULI["Y"], PAULI["Y"])
    assert np.allclose(scipy.linalg.expm(0.25j * math.pi * (XX + YY)), want, atol=1e-14)
    gates = [W.Gate("ROT", (0, 1), theta=-math.pi / 2, paulis="XX"),
             W.Gate("ROT", (0, 1), theta=-math.pi / 2, paulis="YY")]
    assert np.allclose(full_matrix(2, gates), want, atol=1e-14)


# ------------------------------------------------------------------ closed forms

def test_bell_and_ghz():
    psi = oracle.apply_circuit(oracle.zero_state(2), 2, [W.Gate("H", (0,)), W.cnot(0, 1)])
    assert np.allclose(psi, [1 / math.sqrt(2), 0, 0, 1 / math.sqrt(2)], atol=1e-15)
    n = 6
    gates = [W.Gate("H", (0,))] + [W.cnot(q, q + 1) for q in range(n - 1)]
    psi = oracle.apply_circuit(oracle.zero_state(n), n, gates)
    want = np.zeros(1 << n, complex)
    want[0] = want[-1] = 1 / math.sqrt(2)
    assert np.allclose(psi, want, atol=1e-15)


def test_rx_on_zero():
    for th in (0.0, 0.3, 1.7, -2.5, 7.0):
        psi = oracle.apply_circuit(oracle.zero_state(1), 1, [W.Gate("RX", (0,), theta=th)])
        assert np.allclose(psi, [math.cos(th / 2), -1j * math.sin(th / 2)], atol=1e-15)


def bitrev(v, n):
    idx = np.arange(1 << n)
    r = np.zeros_like(idx)
    for b in range(n):
        r |= ((idx >> b) & 1) << (n - 1 - b)
    return v[r]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_qft_equals_scaled_ifft_of_bit_reversal(n):
    # App. "Extending QBIR": apply!(r, QFT) = invorder!, then sqrt(N) * ifft!
    psi = W.haar_state(n, seed=n)
    got = oracle.apply_circuit(psi, n, W.qft(n))
    want = math.sqrt(1 << n) * np.fft.ifft(bitrev(psi, n))
    assert np.allclose(got, want, atol=1e-13)
    # with the final swap network the output is bit-reversed once more
    got_sw = oracle.apply_circuit(psi, n, W.qft(n, swaps=True))
    assert np.allclose(got_sw, bitrev(want, n), atol=1e-13)
    # basis state |x>: amplitudes of modulus 1/sqrt(N)
    x = W.random_basis(n, seed=5)
    b = oracle.apply_circuit(oracle.basis_state(n, x), n, W.qft(n, swaps=True))
    assert np.allclose(np.abs(b), 1 / math.sqrt(1 << n), atol=1e-14)


def test_qft3_listing_and_iqft_dagger():
    rows = []
    import os
    from conftest import ROOT
    with open(os.path.join(ROOT, "tests", "golden", "qft3_listing.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    gates = W.qft(3)
    assert len(gates) == len(rows)
    for g, (name, tq, cq, ang) in zip(gates, rows):
        assert g.name == name and g.locs == (int(tq) - 1,)
        assert g.ctrl_locs == (() if cq == "0" else (int(cq) - 1,))
        if name == "SHIFT":
            assert g.theta == pytest.approx(float(ang), abs=1e-16)
    # iqft = qft' (listing "inverse QFT"): qft then its dagger is the identity
    psi = W.haar_state(3, seed=9)
    back = oracle.apply_dagger(oracle.apply_circuit(psi, 3, gates), 3, gates)
    assert np.allclose(back, psi, atol=1e-14)
    assert np.allclose(full_matrix(3, gates) @ np.conj(full_matrix(3, gates)).T, np.eye(8), atol=1e-14)


def test_hadamard_decomposition_up_to_phase():
    # Listing "gate decomposition": H = Rz(pi/2) Rx(pi/2) Rz(pi/2) up to a global phase
    h = math.pi / 2
    M = full_matrix(1, [W.Gate("RZ", (0,), theta=h), W.Gate("RX", (0,), theta=h),
                        W.Gate("RZ", (0,), theta=h)])
    H = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    ph = M[0, 0] / H[0, 0]
    assert abs(abs(ph) - 1) < 1e-14
    assert np.allclose(M, ph * H, atol=1e-14)


def test_shor_code_restores_input():
    # App. "Symbolic Computation": weight-9 error X,Z,Z,X,Z,Z,X,Z,Z is corrected
    err = [W.Gate(p, (q,)) for q, p in enumerate("XZZXZZXZZ")]
    alpha, beta = 0.6, 0.8j
    psi = np.zeros(1 << 9, complex)
    psi[0], psi[1] = alpha, beta
    out = oracle.apply_circuit(psi, 9, W.shor_circuit(err)).reshape((256, 2))  # [rest][qubit 1]
    rho = out.T @ out.conj()  # reduced density matrix of paper qubit 1 (loc 0)
    v = np.array([alpha, beta])
    assert np.allclose(rho, np.outer(v, v.conj()), atol=1e-14)


# ------------------------------------------------------------------ invariants

def test_norm_and_inverse_identity():
    n = 7
    gates, params = W.variational(n, 3, "ring", seed=4)
    gates = gates + W.qft(n, swaps=True) + [W.toffoli(0, 3, 6), W.Gate("ROT", (1, 5), theta=0.4, paulis="XY")]
    psi = W.haar_state(n, seed=2)
    out = oracle.apply_circuit(psi, n, gates, params)
    assert abs(np.linalg.norm(out) - 1) < 1e-13
    assert np.allclose(oracle.apply_dagger(out, n, gates, params), psi, atol=1e-13)


def test_dagger_of_every_gate_kind_inverts_it():
    # the dagger rules (Sec. "Manipulating Quantum Circuits") for each kind on its
    # own, with and without controls: U^dag U = 1 on a Haar state
    n = 5
    rs = np.random.default_rng(6)
    psi = W.haar_state(n, seed=6)
    kinds = ["I", "X", "Y", "Z", "H", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "SHIFT", "PHASE"]
    gates = [W.Gate(k, (2,), theta=0.77) for k in kinds]
    gates += [W.Gate("SWAP", (1, 3)), W.Gate("ROT", (0, 4), theta=-1.3, paulis="YZ"),
              W.Gate("MATRIX", (3, 1), matrix=scipy.stats.unitary_group.rvs(4, random_state=7))]
    for g in list(gates):
        ctrl = tuple(q for q in range(n) if q not in g.locs)[:2]
        gates.append(W.Gate(g.name, g.locs, ctrl, (1, 0), theta=g.theta, paulis=g.paulis, matrix=g.matrix))
    for g in gates:
        out = oracle.apply_circuit(psi, n, [g])
        back = oracle.apply_dagger(out, n, [g])
        assert np.max(np.abs(back - psi)) < 1e-14, (g.name, g.ctrl_locs)
        if g.name != "I":
            assert np.max(np.abs(out - psi)) > 1e-3, g.name   # the gate itself is not the identity here


def test_single_gate_suite_repetition_invariants():
    n = 5
    psi = W.haar_state(n, seed=11)
    for label, g in W.single_gate_suite(n):
        out = oracle.apply_circuit(psi, n, [g] * 100)
        if g.name in ("X", "H"):
            want = psi  # involutions: 100 applications = identity
        elif g.name == "T":
            want = oracle.apply_circuit(psi, n, [W.Gate("Z", g.locs)])  # T^100 = T^4 = Z
        elif g.name == "RX":
            want = oracle.apply_circuit(psi, n, [W.Gate("RX", g.locs, theta=70.0)])  # Rx(0.7)^100 = Rx(70)
        assert np.allclose(out, want, atol=1e-12), label


# ------------------------------------------------------------------ expectation

def test_expectation_closed_forms_and_dense():
    n = 3
    # basis states: <Z_q> = +-1
    for x in range(8):
        for q in range(n):
            assert oracle.expect(oracle.basis_state(n, x), n, W.z_on(q)) == (1 - 2 * ((x >> q) & 1))
    # heisenberg (periodic) on |000>: each ZZ bond gives 1, XX and YY give 0
    assert oracle.expect(oracle.zero_state(3), 3, W.heisenberg(3)) == pytest.approx(3.0, abs=1e-15)
    # (|0> + i|1>)/sqrt2 has <Y> = 1; |+> has <X> = 1
    assert oracle.expect(np.array([1, 1j]) / math.sqrt(2), 1, [(1.0, ((0, "Y"),))]) == pytest.approx(1.0)
    assert oracle.expect(np.array([1, 1]) / math.sqrt(2), 1, [(1.0, ((0, "X"),))]) == pytest.approx(1.0)
    # random state, random Pauli sums vs the dense kron operator
    rs = np.random.default_rng(5)
    for n in (2, 4, 6):
        psi = W.haar_state(n, seed=n + 100)
        terms = []
        for _ in range(6):
            q = rs.permutation(n)[: rs.integers(1, n + 1)]
            terms.append((float(rs.standard_normal()), tuple((int(l), "XYZ"[rs.integers(3)]) for l in q)))
        O = sum(c * kron_full(n, {l: PAULI[p] for l, p in ops}) for c, ops in terms)
        assert oracle.expect(psi, n, terms) == pytest.approx(float(np.real(psi.conj() @ O @ psi)), abs=1e-13)
        assert np.allclose(oracle.apply_observable(psi, n, terms), O @ psi, atol=1e-13)


def test_pairwise_sum_is_pairwise():
    # a sum whose left fold and pairwise order differ in FP64
    v = np.array([1.0, 1e-16, 1e-16, 1e-16, 1e-16, 1e-16, 1e-16, 1e-16])
    assert oracle.pairwise_sum(v) == (((1.0 + 1e-16) + (1e-16 + 1e-16)) + ((1e-16 + 1e-16) + (1e-16 + 1e-16)))
    x = np.random.default_rng(0).standard_normal(1000)
    assert oracle.pairwise_sum(x) == pytest.approx(math.fsum(x), abs=1e-12)


# ------------------------------------------------------------------ gradients

def test_symad_energy_and_gradient():
    g = read_golden("symad.txt")
    gates, params = W.symad_circuit()
    assert list(params) == [g["alpha"], g["beta"], g["gamma"]]
    loss, grad = oracle.gradient(oracle.zero_state(3), 3, gates, params, W.heisenberg(3))
    assert loss == pytest.approx(g["energy"], rel=1e-15, abs=0)
    want = [g["grad_alpha"], g["grad_beta"], g["grad_gamma"]]
    assert np.allclose(grad, want, rtol=1e-14, atol=0)


def test_adjoint_matches_parameter_shift_on_pauli_rotations():
    n = 4
    gates, params = W.variational(n, 2, "ring", seed=8)
    gates = gates + [W.Gate("ROT", (0, 2), param=len(params), paulis="XZ")]
    params = np.append(params, 0.9)
    terms = W.tfim(n)
    psi0 = oracle.zero_state(n)
    _, grad = oracle.gradient(psi0, n, gates, params, terms)
    assert np.allclose(grad, oracle.shift_gradient(psi0, n, gates, params, terms), atol=1e-12)


def test_adjoint_matches_finite_differences_everywhere():
    n = 5
    rs = np.random.default_rng(12)
    gates = [
        W.Gate("RX", (0,), param=0), W.Gate("RY", (2,), (0,), (1,), param=1),
        W.Gate("SHIFT", (1,), (3,), (0,), param=2), W.Gate("H", (4,)),
        W.Gate("ROT", (1, 4), param=3, paulis="YZ"), W.toffoli(0, 1, 3),
        W.Gate("PHASE", (2,), (4,), (1,), param=4), W.Gate("RZ", (3,), (0, 2), (1, 0), param=5),
        W.Gate("MATRIX", (2, 0), matrix=rand_unitary(2, rs)), W.Gate("RX", (4,), param=0),
    ]
    params = rs.uniform(0, 2 * math.pi, 6)
    psi0 = W.haar_state(n, seed=1)
    terms = W.heisenberg(n) + [(0.3, ((1, "X"),))]
    _, grad = oracle.gradient(psi0, n, gates, params, terms)
    fd = oracle.fd_gradient(psi0, n, gates, params, terms, h=1e-5)
    assert np.allclose(grad, fd, atol=1e-8)


def test_shift_rule_fails_for_controlled_rotation():
    # Eq. shiftrule needs a reflexive generator; control(.., Ry) has generator P1 (x) Y.
    gates, params = W.symad_circuit()
    with pytest.raises(ValueError):
        oracle.shift_gradient(oracle.zero_state(3), 3, gates, params, W.heisenberg(3))


# ------------------------------------------------------------------ sampling

def test_sampling_dyadic_exact():
    n = 3
    probs = np.array([0.5, 0.25, 0.125, 0.125, 0, 0, 0, 0])
    psi = np.sqrt(probs).astype(complex)
    u = np.array([0.0, 0.25, 0.4999999, 0.5, 0.7, 0.75, 0.8, 0.875, 0.9, 0.999999])
    want = [0, 0, 0, 1, 1, 2, 2, 3, 3, 3]  # smallest i with CDF_i > u
    assert list(oracle.sample(psi, n, u)) == want


def test_sampling_crosses_block_levels():
    n = 21  # 2048 level-0 blocks, 2 level-1 blocks
    dim = 1 << n
    support = {5: 0.25, 1500: 0.125, 1_048_575: 0.125, 1_048_576: 0.25, dim - 1: 0.25}
    psi = np.zeros(dim, complex)
    for i, p in support.items():
        psi[i] = math.sqrt(p) * np.exp(1j * i)
    u = np.array([0.1, 0.3, 0.4, 0.55, 0.6, 0.74, 0.8, 0.99])
    cdf_keys = sorted(support)
    cdf = np.cumsum([support[k] for k in cdf_keys])
    want = [cdf_keys[int(np.searchsorted(cdf, x, side="right"))] for x in u]
    assert list(oracle.sample(psi, n, u)) == want


def test_sampling_matches_inverse_cdf_and_histogram():
    n = 10
    psi = W.haar_state(n, seed=21)
    u = W.shot_uniforms(20000, seed=4)[0]
    s = oracle.sample(psi, n, u)
    p = np.abs(psi) ** 2
    ref = np.searchsorted(np.cumsum(p), u * p.sum(), side="right")
    assert np.mean(s == ref) > 0.999  # only rounding ties may differ
    hist = np.bincount(s, minlength=1 << n)
    stat, pval = scipy.stats.chisquare(hist, p / p.sum() * len(u))
    assert pval > 1e-4


def test_collapse():
    psi = W.haar_state(4, seed=3)
    out = oracle.collapse(psi, 4, 9)
    assert abs(abs(out[9]) - 1) < 1e-15 and np.count_nonzero(out) == 1
    assert np.angle(out[9]) == pytest.approx(np.angle(psi[9]))


def test_splitmix64_published_outputs_and_uniforms():
    # the seeded measurement's generator against its published reference outputs
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "splitmix64.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for seed, k, want in rows:
        assert oracle.splitmix64(int(seed), int(k)) == int(want, 16), (seed, k)
    # u = top 53 bits / 2^53: in [0, 1), and draw k of register r is r * nshots + j + 1
    u = oracle.seeded_uniforms(0, 2, 3)
    assert u[0, 0] == (0xE220A8397B1DCDAF >> 11) / 2.0 ** 53
    assert u[0, 2] == (0x06C45D188009454F >> 11) / 2.0 ** 53
    assert u[1, 0] == (oracle.splitmix64(0, 4) >> 11) / 2.0 ** 53
    big = oracle.seeded_uniforms(12345, 4, 5000)
    assert big.min() >= 0.0 and big.max() < 1.0
    # uniformity: chi-square over 20 bins of 20000 draws (p > 1e-4)
    h, _ = np.histogram(big, bins=20, range=(0, 1))
    chi2 = float(np.sum((h - 1000.0) ** 2 / 1000.0))
    assert chi2 < 56.0, chi2
    # seeded sampling = sampling with those uniforms
    n = 5
    psi = W.haar_state(n, seed=2)
    assert (oracle.sample_seeded(psi, n, 7, 64, reg=1) == oracle.sample(psi, n, oracle.seeded_uniforms(7, 2, 64)[1])).all()
