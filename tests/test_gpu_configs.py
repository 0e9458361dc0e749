"""The larger workloads at their full sizes.

- differentiation: n = 20, 100 layers of Rz Rx Rz + CNOT ring (8000 gates, 6000
  angles), transverse-field Ising loss; complex64 forward with checkpoints every
  10 layers and the FP64 uncompute, against the oracle's adjoint gradient at the
  same size; the same circuit shape at n = 10 against parameter shift and finite
  differences on the oracle.
- large: n = 32 (32 GiB) QFT with swap network on a seeded basis state, then a
  depth-20 brickwork of Rz + Haar SU(2) gates and CZs, and the reversible gradient
  of <Z_1> on the tile engine: QFT amplitudes against the closed form at sampled
  indices, norm, light-cone zeros of the gradient; the same pipeline at n = 22
  element by element against the oracle.
"""
import math

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


def diff_gradient(qs, n, depth, dtype, every):
    gates, params = W.variational(n, depth, "ring", seed=0)
    terms = W.tfim(n)
    circ = qs.Circuit(gates, n)
    obs = qs.Observable(terms)
    st = qs.State(n, dtype=dtype)
    st.reset()
    ck = qs.checkpoint_buffer(st, circ, every)
    qs.apply_circuit_ckpt(st, circ, params, every, ck)
    loss, grad = qs.backward(st, circ, params, obs, every, ck)
    return gates, params, terms, loss, grad


def test_differentiation_n10_against_shift_and_fd(qs):
    n, depth = 10, 100
    gates, params, terms, loss, grad = diff_gradient(qs, n, depth, torch.complex128, 10 * (4 * n))
    rl, rg = oracle.gradient(oracle.zero_state(n), n, gates, params, terms)
    assert abs(loss - rl) < 1e-10
    assert np.max(np.abs(grad - rg)) / np.max(np.abs(rg)) < 1e-6
    idx = list(range(0, len(params), 397))
    sub_gates = gates
    shift = {}
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += math.pi / 2
        pm[i] -= math.pi / 2
        shift[i] = 0.5 * (oracle.loss(oracle.zero_state(n), n, sub_gates, pp, terms)
                          - oracle.loss(oracle.zero_state(n), n, sub_gates, pm, terms))
    fd = oracle.fd_gradient(oracle.zero_state(n), n, gates, params, terms, h=1e-5, which=idx)
    scale = np.max(np.abs(rg))
    for i in idx:
        assert abs(grad[i] - shift[i]) / scale < 1e-6
        assert abs(grad[i] - fd[i]) / scale < 1e-6


def test_differentiation_n20_full_size(qs, record_property):
    n, depth = 20, 100
    gates, params, terms, loss, grad = diff_gradient(qs, n, depth, torch.complex64, 10 * (4 * n))
    rl, rg = oracle.gradient(oracle.zero_state(n), n, gates, params, terms)
    err = float(np.max(np.abs(grad - rg)) / np.max(np.abs(rg)))
    record_property("grad_rel_err_c64_forward_fp64_uncompute", err)
    record_property("loss_abs_err", abs(loss - rl))
    print(f"n=20 differentiation: |dloss|={abs(loss - rl):.3e} grad max rel err={err:.3e}")
    # measured on GB300: loss 9.2e-9, gradient 2.5e-6 (the storage rounding of the complex64
    # forward over 100 layers; compensated gate matrices and the FP64 uncompute remove the rest)
    assert abs(loss - rl) < 1e-6
    assert err < 8e-6


def large_pipeline(qs, n, depth, seed=0):
    x = W.random_basis(n, seed=seed)
    qft = W.qft(n, swaps=True)
    bgates, bparams = W.brickwork(n, depth, seed=seed)
    st = qs.State(n, dtype=torch.complex64)
    st.reset([x])
    st.apply_circuit(qs.Circuit(qft, n), tiles=True)
    bcirc = qs.Circuit(bgates, n, nparams=len(bparams))
    st.apply_circuit(bcirc, bparams, tiles=True)
    loss, grad = qs.backward_tiled(st, bcirc, bparams, qs.Observable(W.z_on(0)))
    return x, qft, bgates, bparams, st, loss, grad


def test_large_pipeline_n22_against_oracle(qs):
    n = 22
    x, qft, bgates, bparams, st, loss, grad = large_pipeline(qs, n, 20)
    psi0 = oracle.apply_circuit(oracle.basis_state(n, x), n, qft)
    psiN = oracle.apply_circuit(psi0, n, bgates, bparams)
    assert np.max(np.abs(st.numpy() - psiN)) < 2e-5
    rl, rg = oracle.gradient(psi0, n, bgates, bparams, W.z_on(0))
    err = float(np.max(np.abs(grad - rg)) / np.max(np.abs(rg)))
    print(f"n=22 tile-engine pipeline: loss {abs(loss - rl):.2e} grad {err:.2e}")
    assert abs(loss - rl) < 1e-5
    assert err < 1e-4


def test_large_pipeline_n32_properties(qs):
    n = 32
    x = W.random_basis(n, seed=0)
    st = qs.State(n, dtype=torch.complex64)
    st.reset([x])
    st.apply_circuit(qs.Circuit(W.qft(n, swaps=True), n), tiles=True)
    N = 1 << n
    ks = np.concatenate([np.arange(8), W.rng(1).integers(0, N, 56)]).astype(np.int64)
    got = st.buffer[torch.as_tensor(ks, device="cuda")].cpu().numpy().astype(np.complex128)
    # little-endian QFT with the swap network: |x> -> sum_k e^{2 pi i rev(x) rev(k) / N} |k> / sqrt(N)
    # (rev = n-bit reversal; the oracle pins qft(n)|v> = sqrt(N) IFFT(rev(v)) and the swaps reverse again)
    def rev(v):
        return int(format(int(v), "0%db" % n)[::-1], 2)
    want = np.array([np.exp(2j * np.pi * ((rev(x) * rev(k)) % N) / N) for k in ks]) / math.sqrt(N)
    assert np.max(np.abs(got - want)) * math.sqrt(N) < 1e-3
    bgates, bparams = W.brickwork(n, 20, seed=0)
    bcirc = qs.Circuit(bgates, n, nparams=len(bparams))
    st.apply_circuit(bcirc, bparams, tiles=True)
    nrm = float(torch.sum(torch.abs(st.buffer.to(torch.complex128)) ** 2).item())
    assert abs(nrm - 1.0) < 1e-4
    loss, grad = qs.backward_tiled(st, bcirc, bparams, qs.Observable(W.z_on(0)))
    assert -1.0 <= loss <= 1.0 and np.all(np.isfinite(grad))
    # light cone: an angle on qubit q in layer l can only reach qubit 0 through the
    # CZs of the later layers, at most one qubit per layer
    g = grad.reshape(20, n)
    gmax = float(np.max(np.abs(g)))
    assert gmax > 1e-3
    for layer in range(20):
        later = 20 - layer - 1
        for q in range(n):
            if q > later + 1:
                assert abs(g[layer, q]) < 1e-4 * gmax, (layer, q, g[layer, q])


def test_precise_complex64_apply_against_oracle(qs, record_property):
    # QS_APPLY_PRECISE: compensated 1-qubit gates (fused runs, controls, diagonal and
    # permutation forms) rounded once, against the oracle; its error must not exceed the
    # plain complex64 path's on the same deep circuit
    n, depth = 12, 60
    gates, params = W.variational(n, depth, "ring", seed=9)
    extra = [W.Gate("RY", (3,), (5,), (0,), theta=0.3), W.Gate("SHIFT", (7,), (1,), (1,), theta=1.1),
             W.Gate("T", (2,)), W.Gate("Y", (4,), (9,), (1,)), W.Gate("H", (0,))]
    gates = gates + extra * 20
    circ = qs.Circuit(gates, n, nparams=len(params))
    ref = oracle.apply_circuit(oracle.zero_state(n), n, gates, params)
    errs = {}
    for name, kw in (("plain", {"fused": False}), ("precise", {"precise": True})):
        st = qs.State(n, dtype=torch.complex64)
        st.reset()
        st.apply_circuit(circ, params, **kw)
        errs[name] = float(np.max(np.abs(st.numpy() - ref)))
    record_property("state_abs_err", errs)
    print(f"complex64 n={n}, {len(gates)} gates: max|dpsi| plain {errs['plain']:.2e} precise {errs['precise']:.2e}")
    assert errs["precise"] < 2e-6
    assert errs["precise"] <= errs["plain"]


def _diag_perm_sections(n, reps, seed):
    """Gate runs whose fused blocks are diagonal (Rz, controlled phases, CZ, T) and
    phased permutations (CNOT, SWAP, Y, Toffoli, S, phase), plus one dense run."""
    r = W.rng(seed)
    diag, perm = [], []
    for _ in range(reps):
        q = int(r.integers(0, n - 1))
        diag += [W.Gate("RZ", (q,), theta=float(r.uniform(0, 6.3))), W.Gate("Z", (q + 1,), (q,), (1,)),
                 W.Gate("SHIFT", (q,), (q + 1,), (1,), theta=float(r.uniform(0, 6.3))), W.Gate("T", (q + 1,)),
                 W.Gate("PHASE", (q,), theta=float(r.uniform(0, 6.3)))]
        c = int(r.integers(0, n - 2))
        perm += [W.cnot(c, c + 1), W.Gate("SWAP", (c + 1, c + 2)), W.Gate("Y", (c,)), W.toffoli(c, c + 1, c + 2),
                 W.Gate("S", (c + 2,)), W.Gate("SHIFT", (c + 1,), theta=float(r.uniform(0, 6.3)))]
    return diag, perm


@pytest.mark.parametrize("kind", ["dense", "diagonal", "permutation"])
def test_precise_blocks_against_oracle(qs, kind, record_property):
    # QS_APPLY_PRECISE with QS_APPLY_BLOCKS: every fused block (dense, diagonal or phased
    # permutation of up to 5 qubits) applied with its FP64 matrix as FP32 hi + lo, each
    # output rounded once; the error must stay at the storage-rounding level and not
    # exceed the plain block path's
    n = 12
    if kind == "dense":
        gates, params = W.brickwork(n, 40, seed=4)
    else:
        diag, perm = _diag_perm_sections(n, 150, seed=5)
        gates, params = (diag if kind == "diagonal" else perm), np.zeros(0)
    circ = qs.Circuit(gates, n, nparams=len(params))
    psi_in = W.haar_state(n, seed=6)
    ref = oracle.apply_circuit(psi_in, n, gates, params)
    errs = {}
    for name, kw in (("plain", {}), ("precise", {"precise": True})):
        st = qs.State(n, dtype=torch.complex64)
        st.upload(psi_in)
        st.apply_circuit(circ, params, blocks=5, **kw)
        errs[name] = float(np.max(np.abs(st.numpy() - ref)))
    record_property("state_abs_err", errs)
    print(f"complex64 {kind} blocks n={n}, {len(gates)} gates: max|dpsi| plain {errs['plain']:.2e} "
          f"precise {errs['precise']:.2e}")
    assert errs["precise"] < 1e-6
    assert errs["precise"] <= errs["plain"]
