"""Faithful gradients (Sec. "Forward Mode", Eq. shiftrule) on the GPU against
the oracle.  Exact mode: the shift-rule gradient equals the oracle's shift-rule
and reversible-adjoint gradients.  Shot mode (complex128): the oracle runs the
same contract (groups of qubit-wise commuting terms in order of first
appearance, X -> H, Y -> S^dag then H, the deterministic sampler with the same
uniforms, parity counts) and must reach the same estimate to rounding of the
final FP64 sums (sample indices are bit-exact; one differing sample would move
an estimate by >= 2/nshots).  Complex64 shots: within 6 standard errors of the
exact gradient."""
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


def letters(term):
    c, ops = term
    return c, {q: p for q, p in ops}


def groups_of(terms):
    """The grouping contract, written from its definition."""
    gs, const = [], 0.0
    for t, term in enumerate(terms):
        c, ops = letters(term)
        if not ops:
            const += c
            continue
        for g in gs:
            if all(g["basis"].get(q, p) == p for q, p in ops.items()):
                g["basis"].update(ops)
                g["terms"].append(t)
                break
        else:
            gs.append({"basis": dict(ops), "terms": [t]})
    return gs, const


def oracle_shot_expect(psi, n, terms, u):
    gs, const = groups_of(terms)
    acc = 0.0
    for g, grp in enumerate(gs):
        rot = []
        for q, p in sorted(grp["basis"].items()):
            if p == "Y":
                rot.append(W.Gate("SDG", (q,)))
            if p in ("X", "Y"):
                rot.append(W.Gate("H", (q,)))
        x = oracle.sample(oracle.apply_circuit(psi, n, rot), n, u[g])
        ga = 0.0
        for t in grp["terms"]:
            c, ops = letters(terms[t])
            supp = sum(1 << q for q in ops)
            cnt = int(np.sum(1 - 2 * (np.array([bin(int(v) & supp).count("1") & 1 for v in x]))))
            ga += c * (cnt / len(x))
        acc += ga
    return acc + const


def mixed_terms(n):
    return [(0.7, ((0, "Z"), (1, "Z"))), (-0.4, ((2, "X"),)), (0.3, ((1, "Y"), (3, "Y"))),
            (0.25, ((0, "X"), (3, "Z"))), (1.5, ()), (-0.2, ((2, "Z"),)), (0.6, ((n - 1, "X"), (0, "Y")))]


def test_groups_match_the_library(qs):
    n = 6
    for terms in (mixed_terms(n), W.tfim(n, 1.0), W.heisenberg(n)):
        gs, _ = groups_of(terms)
        assert qs.observable_groups(qs.Observable(terms)) == len(gs)


def test_shot_expectation_matches_oracle_contract(qs):
    n = 7
    gates, params = W.variational(n, 2, "ring", seed=3)
    psi = oracle.apply_circuit(oracle.zero_state(n), n, gates, params)
    for terms in (mixed_terms(n), W.tfim(n, 1.0)):
        obs = qs.Observable(terms)
        G = qs.observable_groups(obs)
        nshots, nreg = 2000, 3
        u = W.shot_uniforms(nshots, seed=11, nreg=G * nreg).reshape(G, nreg, nshots)
        st = qs.State(n, dtype=torch.complex128, nbatch=nreg)
        st.upload(np.tile(psi, nreg))
        got = qs.shot_expect(st, obs, u)
        for r in range(nreg):
            want = oracle_shot_expect(psi, n, terms, u[:, r, :])
            assert abs(got[r] - want) < 1e-12, (r, got[r], want)
        # and the estimates scatter around the exact value
        exact = oracle.expect(psi, n, terms)
        assert abs(np.mean(got) - exact) < 6 * sum(abs(c) for c, _ in terms) / math.sqrt(nshots * nreg)


def test_exact_shift_rule_gradient(qs):
    n = 6
    gates, params = W.variational(n, 2, "ring", seed=5)
    terms = W.tfim(n, 1.0)
    circ = qs.Circuit(gates, n)
    obs = qs.Observable(terms)
    for dt, tol in ((torch.complex128, 1e-10), (torch.complex64, 2e-5)):
        g = qs.faithful_gradient(circ, params, obs, dtype=dt)
        want = oracle.shift_gradient(oracle.zero_state(n), n, gates, params, terms)
        _, adj = oracle.gradient(oracle.zero_state(n), n, gates, params, terms)
        scale = np.max(np.abs(want))
        assert np.max(np.abs(g - want)) / scale < tol, dt
        assert np.max(np.abs(g - adj)) / scale < tol, dt


def test_shot_shift_rule_gradient_matches_oracle(qs):
    n = 5
    gates, params = W.variational(n, 1, "ladder", seed=2)
    terms = mixed_terms(n)
    circ = qs.Circuit(gates, n)
    obs = qs.Observable(terms)
    P = len(params)
    G = qs.observable_groups(obs)
    nshots = 512
    u = W.shot_uniforms(nshots, seed=21, nreg=G * 2 * P).reshape(G, 2 * P, nshots)
    got = qs.faithful_gradient(circ, params, obs, dtype=torch.complex128, nshots=nshots, uniforms=u)
    want = np.zeros(P)
    for k in range(P):
        pp, pm = np.array(params, dtype=float), np.array(params, dtype=float)
        pp[k] += math.pi / 2
        pm[k] -= math.pi / 2
        ep = oracle_shot_expect(oracle.apply_circuit(oracle.zero_state(n), n, gates, pp), n, terms, u[:, 2 * k, :])
        em = oracle_shot_expect(oracle.apply_circuit(oracle.zero_state(n), n, gates, pm), n, terms, u[:, 2 * k + 1, :])
        want[k] = 0.5 * (ep - em)
    assert np.max(np.abs(got - want)) < 1e-12
    # complex64 through the batched engine: statistically consistent with the exact gradient
    exact = oracle.shift_gradient(oracle.zero_state(n), n, gates, params, terms)
    n64 = 20000
    u64 = W.shot_uniforms(n64, seed=22, nreg=G * 2 * P).reshape(G, 2 * P, n64)
    g64 = qs.faithful_gradient(circ, params, obs, dtype=torch.complex64, nshots=n64, uniforms=u64)
    se = sum(abs(c) for c, _ in terms) / math.sqrt(n64)
    assert np.max(np.abs(g64 - exact)) < 6 * se


def test_shift_rule_rejects_controlled_and_shared_parameters(qs):
    from paper_1912_10877_gb300 import _native as N
    n = 4
    obs = qs.Observable(W.zz_chain(n))
    bad1 = qs.Circuit([W.Gate("RX", (0,), (1,), (1,), param=0)], n)
    bad2 = qs.Circuit([W.Gate("RX", (0,), param=0), W.Gate("RY", (1,), param=0)], n)
    for c in (bad1, bad2):
        with pytest.raises(N.QsimError) as e:
            qs.faithful_gradient(c, [0.3], obs)
        assert e.value.code == N.QS_EUNSUPPORTED


def kernel_matrix(n, sigma):
    x = np.arange(1 << n, dtype=float)
    return np.exp(-(x[:, None] - x[None, :]) ** 2 / (2 * sigma * sigma))


def oracle_mmd(n, gates, params, q, sigma, nshots=0, u=None):
    """Loss and shift-rule gradient from the oracle's distributions (exact) or from the
    oracle's samples with the same uniforms (register order: 2k +, 2k+1 -, 2P unshifted)."""
    P = len(params)
    K = kernel_matrix(n, sigma)
    dists = []
    for r in range(2 * P + 1):
        pr = np.array(params, dtype=float)
        if r < 2 * P:
            pr[r // 2] += -math.pi / 2 if r % 2 else math.pi / 2
        psi = oracle.apply_circuit(oracle.zero_state(n), n, gates, pr)
        if nshots:
            x = oracle.sample(psi, n, u[r])
            dists.append(np.bincount(np.asarray(x, dtype=np.int64), minlength=1 << n) / nshots)
        else:
            dists.append(np.abs(psi) ** 2)
    p = dists[-1]
    loss = p @ K @ p - 2 * p @ K @ q + q @ K @ q
    w = K @ p - K @ q
    grad = np.array([(dists[2 * k] - dists[2 * k + 1]) @ w for k in range(P)])
    return loss, grad


@pytest.mark.parametrize("sigma", [0.7, 3.0])
def test_mmd_gradient_exact_and_shots(qs, sigma):
    n = 5
    gates, params = W.variational(n, 1, "ladder", seed=4)
    rs = np.random.default_rng(5)
    q = rs.random(1 << n)
    q /= q.sum()
    circ = qs.Circuit(gates, n)
    P = len(params)
    loss, g = qs.mmd_gradient(circ, params, q, sigma)
    wl, wg = oracle_mmd(n, gates, params, q, sigma)
    assert abs(loss - wl) < 1e-12 and np.max(np.abs(g - wg)) < 1e-12
    nshots = 400
    u = W.shot_uniforms(nshots, seed=9, nreg=2 * P + 1)
    loss, g = qs.mmd_gradient(circ, params, q, sigma, nshots=nshots, uniforms=u)
    wl, wg = oracle_mmd(n, gates, params, q, sigma, nshots, u)
    assert abs(loss - wl) < 1e-12 and np.max(np.abs(g - wg)) < 1e-12
    # complex64, exact distributions from FP32 amplitudes
    loss64, g64 = qs.mmd_gradient(circ, params, q, sigma, dtype=torch.complex64)
    wl, wg = oracle_mmd(n, gates, params, q, sigma)
    assert abs(loss64 - wl) < 1e-5 and np.max(np.abs(g64 - wg)) < 1e-5
