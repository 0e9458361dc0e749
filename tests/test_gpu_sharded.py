"""GPU parity of the level-1 entry points (qs_state_copy / inner / axpy) and of
the qubit-sharded register with its shards as libqsim registers on one GPU (all
shards in one process; exchanges are device copies).  Tolerances: complex128
1e-12 on amplitudes and expectations, 1e-10 relative on gradients; complex64
2e-5 on amplitudes, 1e-4 on expectations and relative gradients (FP32 states
through every gate)."""
import numpy as np
import pytest

import oracle
import workloads as W
from test_sharded_cpu import mixed_circuit

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TDT = {"c64": torch.complex64, "c128": torch.complex128}
NPT = {"c64": np.complex64, "c128": np.complex128}
TOL = {"c64": dict(state=2e-5, expect=1e-4, grad=1e-4), "c128": dict(state=1e-12, expect=1e-12, grad=1e-10)}


@pytest.fixture(scope="module")
def qs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10877_gb300 import qsim
    oracle.build()
    return qsim


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_level1_ops_against_numpy(qs, dt):
    counts = [3, 9, 12, 1]
    rs = np.random.default_rng(7)
    total = sum(1 << c for c in counts)
    xa = (rs.standard_normal(total) + 1j * rs.standard_normal(total)).astype(NPT[dt])
    xb = (rs.standard_normal(total) + 1j * rs.standard_normal(total)).astype(NPT[dt])
    a = qs.State(counts, dtype=TDT[dt]).upload(xa)
    b = qs.State(counts, dtype=TDT[dt]).upload(xb)
    off = np.cumsum([0] + [1 << c for c in counts])
    got = a.inner(b)
    for r in range(len(counts)):
        u = xa[off[r]:off[r + 1]].astype(np.complex128)
        v = xb[off[r]:off[r + 1]].astype(np.complex128)
        want = np.vdot(u, v)   # products of the stored values are exact in FP64
        assert abs(got[r] - want) <= 1e-12 * np.linalg.norm(u) * np.linalg.norm(v), r
    alpha = 0.37 - 1.21j
    b.axpy(alpha, a)
    al = complex(np.complex64(alpha)) if dt == "c64" else alpha
    want = xb.astype(np.complex128) + al * xa.astype(np.complex128)
    eps = 2e-6 if dt == "c64" else 1e-14
    assert np.max(np.abs(b.numpy() - want)) <= eps * np.max(np.abs(want))
    c = qs.State(counts, dtype=TDT[dt])
    c.copy_from(a)
    assert np.array_equal(c.numpy(), xa)


@pytest.mark.parametrize("dt", ["c64", "c128"])
@pytest.mark.parametrize("n,nglobal", [(8, 2), (11, 3)])
def test_sharded_register_against_oracle(qs, dt, n, nglobal):
    from paper_1912_10877_gb300.sharded import ShardedState
    gates, params = mixed_circuit(n, seed=n + nglobal)
    circ = qs.Circuit(gates, n)
    psi0 = W.haar_state(n, seed=3)
    terms = W.tfim(n) + W.heisenberg(n)[:6] + [(0.3, ((0, "Y"), (n - 1, "X"), (n - 2, "Z")))]
    sh = ShardedState(n, nglobal, TDT[dt])
    sh.upload(psi0)
    sh.apply_circuit(circ, params)
    want = oracle.apply_circuit(psi0, n, gates, params)
    tol = TOL[dt]
    assert sh.exchanges > 0
    assert np.max(np.abs(sh.gather() - want)) < tol["state"]
    assert abs(sh.expect(terms) - oracle.expect(want, n, terms)) < tol["expect"]
    loss, grad = sh.backward(circ, params, terms)
    wloss, wgrad = oracle.gradient(psi0, n, gates, params, terms)
    assert abs(loss - wloss) < tol["expect"]
    assert np.max(np.abs(grad - wgrad)) / np.max(np.abs(wgrad)) < tol["grad"]
    assert np.max(np.abs(sh.gather() - psi0)) < 10 * tol["state"]


def test_sharded_variational_n22_against_oracle(qs):
    """Four shards of 2^20 complex64 amplitudes (runs of up to 2^20 per exchange):
    a ring variational circuit, whole-register parity and the TFIM energy."""
    from paper_1912_10877_gb300.sharded import ShardedState
    n = 22
    gates, params = W.variational(n, 2, entangler="ring", seed=1)
    circ = qs.Circuit(gates, n)
    sh = ShardedState(n, 2, torch.complex64)
    sh.apply_circuit(circ, params)
    want = oracle.apply_circuit(oracle.zero_state(n), n, gates, params)
    assert sh.exchanges > 0
    assert np.max(np.abs(sh.gather() - want)) < 2e-5
    terms = W.tfim(n)
    assert abs(sh.expect(terms) - oracle.expect(want, n, terms)) < 1e-4


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_sharded_sampling(qs, dt):
    # shard drawn from the shard weights (FP64 inner products on the GPU), index
    # from the library's sampler inside the shard, mapped back to the logical
    # index: checked step by step against the oracle's sampler on each shard
    # (promoted to FP64), by a chi-square test against |psi|^2, and on basis states
    import scipy.stats
    from paper_1912_10877_gb300.sharded import ShardedState
    n, nglobal = 11, 3
    gates, params = mixed_circuit(n, seed=n + nglobal)
    sh = ShardedState(n, nglobal, TDT[dt])
    sh.upload(W.haar_state(n, seed=4))
    sh.apply_circuit(qs.Circuit(gates, n), params)
    assert sh.exchanges > 0
    u = W.shot_uniforms(4000, seed=6)[0]
    got = sh.measure(u)
    w = [v.inner(v).real for v in sh.vecs["psi"]]
    shards = [v.numpy().astype(np.complex128) for v in sh.vecs["psi"]]
    total = 0.0
    for x in w:
        total = total + x
    want = []
    for ui in u:
        t = ui * total
        acc, s = 0.0, 0
        while acc + w[s] <= t:
            acc, s = acc + w[s], s + 1
        sub = min((t - acc) / w[s], np.nextafter(1.0, 0.0))
        p = (s << sh.L) | int(oracle.sample(shards[s], sh.L, [sub])[0])
        want.append(sum(((p >> sh.pos[q]) & 1) << q for q in range(n)))
    assert np.array_equal(got, np.array(want))
    prob = np.abs(sh.gather().astype(np.complex128)) ** 2
    shots = sh.measure(W.shot_uniforms(60000, seed=7)[0])
    counts = np.bincount(shots, minlength=1 << n)
    keep = prob * len(shots) >= 5
    stat = scipy.stats.chisquare(counts[keep], prob[keep] / prob[keep].sum() * counts[keep].sum())
    assert stat.pvalue > 1e-4, stat
    sh.reset(0b10110011101)
    assert np.all(sh.measure(W.shot_uniforms(64, seed=8)[0]) == 0b10110011101)
