"""Host logic of the qubit-sharded register (paper_1912_10877_gb300.sharded) on
CPU: the global/local qubit map, the pairwise half-shard exchanges, control
predicates and diagonal restriction on global qubits, expectation values with
global Z signs, the gate-by-gate reversible backward with one all-reduce
of the gradient, and measurement (shard drawn from the shard weights, index
from the shard's sampler, physical index mapped back to the logical one).  Shards here are FP64 host vectors whose local operations are
oracle calls, so these tests check the sharding against the oracle's
whole-register results; exchanges run in one process (every shard local) and
across gloo ranks (world size 2: shards paired inside a rank and across
ranks)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads as W

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1912_10877_gb300 import build as B
    B.build()
    oracle.build()


class OracleShard:
    """A shard of 2^L FP64 amplitudes; every local operation is an oracle call."""

    def __init__(self, L, dtype):
        self.n = L
        self.t = torch.zeros(1 << L, dtype=torch.complex128)
        self.a = self.t.numpy()

    def flat(self):
        return torch.view_as_real(self.t).view(-1)

    def reset(self, x=None):
        self.a[:] = 0
        self.a[0 if x is None else int(x)] = 1

    def zero(self):
        self.a[:] = 0

    def apply_matrix(self, U, locs, ctrl_locs=(), ctrl_vals=()):
        g = W.Gate("MATRIX", tuple(locs), tuple(ctrl_locs), tuple(ctrl_vals), matrix=np.asarray(U))
        self.a[:] = oracle.apply_circuit(self.a, self.n, [g])

    def copy_from(self, other):
        self.a[:] = other.a

    def inner(self, other):
        return complex(np.vdot(self.a, other.a))

    def axpy(self, alpha, other):
        self.a += alpha * other.a

    def expect(self, terms):
        return oracle.expect(self.a, self.n, terms)

    def upload(self, amps):
        self.a[:] = amps

    def numpy(self):
        return self.a.copy()

    def measure(self, u):
        return oracle.sample(self.a, self.n, u)

    def apply_pauli(self, p, P):
        self.a[:] = oracle.apply_circuit(self.a, self.n, [W.Gate(P, (int(p),))])

    def adjoint_step(self, lam, gate, params, grad):
        oracle.adjoint_step(self.a, lam.a, self.n, gate, params, grad)

    @staticmethod
    def new_grad(nparams):
        return np.zeros(max(1, nparams))

    @staticmethod
    def grad_host(buf):
        return buf


def mixed_circuit(n, seed):
    """Gates touching global qubits in every way the sharding distinguishes."""
    rs = np.random.default_rng(seed)
    top, mid = n - 1, n // 2
    g = [W.Gate("H", (top,)), W.Gate("RX", (top - 1,), param=0), W.cnot(top, 0), W.cnot(0, top),
         W.Gate("RY", (1,), (top,), (1,), param=1), W.Gate("RY", (top,), (0,), (0,), param=2),
         W.Gate("T", (top,)), W.Gate("SHIFT", (top - 1,), (top,), (1,), param=3),
         W.Gate("RZ", (top,), param=4), W.Gate("Z", (top - 1,), (top,), (1,)),
         W.toffoli(top, top - 1, 0), W.Gate("SWAP", (0, top)), W.Gate("SWAP", (top, top - 1)),
         W.Gate("ROT", (top, mid), paulis="XY", param=5), W.Gate("ROT", (top - 1, top), paulis="ZZ", param=6),
         W.Gate("PHASE", (2,), (top,), (1,), param=7),
         W.Gate("MATRIX", (top, 1, top - 1), matrix=_unitary(8, rs)),
         W.Gate("Y", (top - 1,), (top, mid), (1, 0)), W.Gate("RX", (mid,), (top - 1,), (1,), param=8)]
    for layer in range(2):
        for q in range(n):
            g.append(W.Gate("RZ", (q,), param=9 + 3 * (layer * n + q)))
            g.append(W.Gate("RX", (q,), param=10 + 3 * (layer * n + q)))
            g.append(W.Gate("RZ", (q,), param=11 + 3 * (layer * n + q)))
        for q in range(n - 1):
            g.append(W.cnot(q, q + 1))
        g.append(W.cnot(n - 1, 0))
    params = rs.uniform(0, 2 * np.pi, 9 + 6 * n)
    return g, params


def _unitary(d, rs):
    z = rs.normal(size=(d, d)) + 1j * rs.normal(size=(d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def run_checks(n, nglobal, group=None):
    """Forward state, <O> and gradient of the sharded register against the oracle."""
    from paper_1912_10877_gb300 import qsim
    from paper_1912_10877_gb300.sharded import ShardedState
    gates, params = mixed_circuit(n, seed=n + nglobal)
    circ = qsim.Circuit(gates, n)
    psi0 = W.haar_state(n, seed=3)
    terms = W.tfim(n) + W.heisenberg(n)[:6] + [(0.3, ((0, "Y"), (n - 1, "X"), (n - 2, "Z")))]
    sh = ShardedState(n, nglobal, torch.complex128, group=group, backend=OracleShard)
    sh.upload(psi0)
    sh.apply_circuit(circ, params)
    want = oracle.apply_circuit(psi0, n, gates, params)
    out = {"state": np.max(np.abs(sh.gather() - want))}
    out["expect"] = abs(sh.expect(terms) - oracle.expect(want, n, terms))
    loss, grad = sh.backward(circ, params, terms)
    wloss, wgrad = oracle.gradient(psi0, n, gates, params, terms)
    out["loss"] = abs(loss - wloss)
    out["grad"] = np.max(np.abs(grad - wgrad)) / np.max(np.abs(wgrad))
    out["uncompute"] = np.max(np.abs(sh.gather() - psi0))
    out["exchanges"] = sh.exchanges
    return out


@pytest.mark.parametrize("n,nglobal", [(6, 1), (6, 2), (7, 3)])
def test_one_process_all_shards_local(n, nglobal):
    r = run_checks(n, nglobal)
    assert r["exchanges"] > 0
    for k in ("state", "expect", "loss", "grad", "uncompute"):
        assert r[k] < TOL, (k, r[k])


def test_reset_and_map_after_exchanges():
    from paper_1912_10877_gb300.sharded import ShardedState
    n = 6
    sh = ShardedState(n, 2, torch.complex128, backend=OracleShard)
    sh.reset(0b101101)
    sh.apply_matrix(np.array([[0, 1], [1, 0]]), [n - 1])          # X on a global qubit: one exchange
    assert sh.exchanges == 1 and sh.pos[n - 1] < sh.L
    sh.reset(0b000011)                                             # the map persists; reset follows it
    want = np.zeros(1 << n, np.complex128)
    want[0b000011] = 1
    assert np.array_equal(sh.gather(), want)


def test_global_diagonal_and_control_move_no_data():
    from paper_1912_10877_gb300.sharded import ShardedState
    n = 6
    sh = ShardedState(n, 2, torch.complex128, backend=OracleShard)
    psi0 = W.haar_state(n, seed=5)
    sh.upload(psi0)
    gates = [W.Gate("T", (n - 1,)), W.Gate("SHIFT", (n - 2,), (n - 1,), (1,), theta=0.3),
             W.Gate("RZ", (n - 1,), theta=1.1), W.Gate("H", (0,), (n - 1, n - 2), (1, 0)),
             W.Gate("RX", (1,), (n - 2,), (1,), theta=0.4)]
    for g in gates:
        sh.apply(g)
    assert sh.exchanges == 0
    assert np.max(np.abs(sh.gather() - oracle.apply_circuit(psi0, n, gates))) < TOL


def sampled_register(n, nglobal, group=None):
    from paper_1912_10877_gb300 import qsim
    from paper_1912_10877_gb300.sharded import ShardedState
    gates, params = mixed_circuit(n, seed=n + nglobal)
    sh = ShardedState(n, nglobal, torch.complex128, group=group, backend=OracleShard)
    sh.upload(W.haar_state(n, seed=4))
    sh.apply_circuit(qsim.Circuit(gates, n), params)
    return sh


def two_level_reference(sh, u):
    """The sharded sampling rule written out on the gathered physical shards."""
    psi = sh.gather()
    phys = np.empty_like(psi)
    phys[sh._perm()] = psi
    shards = phys.reshape(sh.nshards, -1)
    w = [float(np.vdot(v, v).real) for v in shards]
    total = 0.0
    for x in w:
        total = total + x
    out = []
    for ui in u:
        t = ui * total
        acc = 0.0
        for s_, ws in enumerate(w):
            if acc + ws > t:
                break
            acc = acc + ws
        sub = min((t - acc) / w[s_], np.nextafter(1.0, 0.0))
        i = int(oracle.sample(shards[s_], sh.L, [sub])[0])
        p = (s_ << sh.L) | i
        out.append(sum(((p >> sh.pos[q]) & 1) << q for q in range(sh.n)))
    return np.array(out, np.int64)


@pytest.mark.parametrize("n,nglobal", [(7, 2), (8, 3)])
def test_sampling_follows_the_two_level_rule(n, nglobal):
    sh = sampled_register(n, nglobal)
    assert sh.exchanges > 0 and sh.pos != list(range(n))
    u = W.shot_uniforms(3000, seed=n)[0]
    assert np.array_equal(sh.measure(u), two_level_reference(sh, u))


def test_sampling_distribution_and_basis_states():
    import scipy.stats
    from paper_1912_10877_gb300.sharded import ShardedState
    n = 6
    sh = sampled_register(n, 2)
    p = np.abs(sh.gather()) ** 2
    shots = sh.measure(W.shot_uniforms(40000, seed=9)[0])
    counts = np.bincount(shots, minlength=1 << n)
    keep = p * len(shots) >= 5
    stat = scipy.stats.chisquare(counts[keep], p[keep] / p[keep].sum() * counts[keep].sum())
    assert stat.pvalue > 1e-4, stat
    assert np.all(p[shots] > 0)
    b = ShardedState(n, 2, torch.complex128, backend=OracleShard)
    b.apply_matrix(np.array([[0, 1], [1, 0]]), [n - 1])   # moves the map
    b.reset(0b110101)
    assert np.all(b.measure(W.shot_uniforms(50, seed=1)[0]) == 0b110101)
    one = ShardedState(n, 0, torch.complex128, backend=OracleShard)
    one.upload(W.haar_state(n, seed=2))
    u = W.shot_uniforms(200, seed=3)[0]
    assert np.array_equal(one.measure(u), oracle.sample(W.haar_state(n, seed=2), n, u))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, nglobal, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r = run_checks(n, nglobal)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([r[k] for k in ("state", "expect", "loss", "grad", "uncompute", "exchanges")]))
    finally:
        dist.destroy_process_group()


def _sample_worker(rank, world, port, n, nglobal, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sh = sampled_register(n, nglobal)
        np.save(os.path.join(out_dir, f"s{rank}.npy"), sh.measure(W.shot_uniforms(2000, seed=5)[0]))
    finally:
        dist.destroy_process_group()


def test_gloo_world_two_sampling(tmp_path):
    n, nglobal, world = 7, 2, 2
    mp.start_processes(_sample_worker, args=(world, free_port(), n, nglobal, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    want = sampled_register(n, nglobal).measure(W.shot_uniforms(2000, seed=5)[0])
    for rank in range(world):
        assert np.array_equal(np.load(tmp_path / f"s{rank}.npy"), want), rank


@pytest.mark.parametrize("n,nglobal", [(6, 1), (7, 2)])
def test_gloo_world_two(tmp_path, n, nglobal):
    world = 2
    mp.start_processes(_worker, args=(world, free_port(), n, nglobal, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        got = np.load(tmp_path / f"r{rank}.npy")
        assert np.all(got[:5] < TOL), (rank, got)
        assert got[5] > 0
