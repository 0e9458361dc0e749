"""Qubit-sharded state vector: one 2^n-amplitude register split into 2^g shards.

A register too large for one device is cut by its top g physical qubits (the
"global" qubits): shard s holds the 2^L amplitudes (L = n - g) whose physical
index has s in its top g bits.  Shards live in the processes of a
torch.distributed group (NCCL between GPUs, gloo on CPU), 2^g / world shards
per process; with no group every shard is local.

Which logical qubit sits at which physical bit is a permutation kept on the
host (``pos`` / ``who``), identical on every rank.  Gates follow the general
instruction of Sec. "Instructions on Quantum Registers" / Sec. "Performance":
  * a control on a global qubit is a predicate on the shard index: shards
    whose bit differs skip the gate, the others drop the control;
  * a diagonal gate never moves data: on each shard its diagonal is restricted
    to the shard's values of the global targets (a scalar when every target is
    global);
  * any other gate first brings its global targets to local bits: physical
    local bit l and global bit j are exchanged by swapping, between shard s and
    shard s ^ 2^j, the half of each shard whose bit l differs from the shard's
    bit j (one pairwise exchange of half the shard, 2^(L-1) amplitudes each way),
    after which the two logical qubits trade places in the map.  The local bit
    given up is the highest one not needed by the gate, so the halves are
    contiguous runs of at least 2^(L-1-k) amplitudes.
Expectation values (Sec. "Forward Mode") localise the X / Y qubits of each
Pauli string the same way and read a global Z as the sign (-1)^bit of the
shard; the per-shard sums are added with one all-reduce.  The reversible
backward (Sec. "Reverse Mode", Eq. apply-back) runs gate by gate on complex128
working copies of psi and lambda = O psi, which share the map: a
parameterised gate has its targets localised and then, on every shard whose
global controls match, one library step (qs_adjoint_step) adds
2 c Im<lambda|(P_ctrl (x) H) psi> to a device gradient and uncomputes both
states by U^dagger in FP64; other gates are uncomputed by U^dagger from the
library.  The gradient is read back and added over the ranks once, at the end.
Measurement (Sec. "Instructions on Quantum Registers", measure) draws a shard
from the shard weights P_s = <psi_s|psi_s> (one all-reduce) with the library's
shard walk (qs_sample_shards), then an index inside it with the shard's own
sampler and the uniform that walk returns, and maps the physical index back to
the logical one.

Every local operation and all of the method's arithmetic is a call into
libqsim.so (``qsim.State`` and the level-1 entry points); this module only
plans exchanges, predicates and which entries of a library-computed diagonal
a shard keeps, and moves shard halves with ``torch.distributed``
point-to-point transfers (across processes) or device copies (inside one).  ``backend`` lets a caller supply shards of another kind
with the same methods (used by the CPU multi-process tests of this logic).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import _native as N
from . import qsim


class LibShard:
    """One shard as a libqsim register on the current CUDA device."""

    def __init__(self, nqubits: int, dtype):
        self.n = nqubits
        self.st = qsim.State(nqubits, dtype=dtype)

    def flat(self) -> torch.Tensor:
        """The amplitudes as a flat real tensor (re, im interleaved)."""
        return torch.view_as_real(self.st.buffer).view(-1)

    def reset(self, x=None):
        self.st.reset(x)

    def zero(self):
        self.st.reset()
        self.st.apply_matrix(np.zeros((2, 2), np.complex128), [0])

    def apply_matrix(self, U, locs, ctrl_locs=(), ctrl_vals=()):
        self.st.apply_matrix(U, list(locs), list(ctrl_locs), list(ctrl_vals))

    def copy_from(self, other: "LibShard"):
        self.st.copy_from(other.st)   # the dtypes may differ (widened or rounded by the library)

    def apply_pauli(self, p: int, P: str):
        """The Pauli P on local bit p (the library's X / Y / Z gate)."""
        loc = N.i32([p])
        N.check(N.lib().qs_apply_named(self.st.handle, N.GATE_KIND[P], 1, loc, N.i32([]), 0, N.i32([]),
                                       N.i32([]), 0.0))

    def adjoint_step(self, lam: "LibShard", gate, params, grad: torch.Tensor):
        """One gate of the reversible adjoint on this shard (psi) and lam, both
        complex128, gate on local bits (qs_adjoint_step)."""
        qsim.adjoint_step(self.st, lam.st, gate, params, grad)

    @staticmethod
    def new_grad(nparams: int) -> torch.Tensor:
        return torch.zeros(max(1, nparams), dtype=torch.float64, device="cuda")

    @staticmethod
    def grad_host(buf: torch.Tensor) -> np.ndarray:
        return buf.cpu().numpy()

    def inner(self, other: "LibShard") -> complex:
        return complex(self.st.inner(other.st)[0])

    def axpy(self, alpha, other: "LibShard"):
        self.st.axpy(alpha, other.st)

    def expect(self, terms) -> float:
        return float(self.st.expect(qsim.Observable(terms))[0])

    def upload(self, amps):
        self.st.upload(amps)

    def numpy(self) -> np.ndarray:
        return self.st.numpy()

    def measure(self, u) -> np.ndarray:
        """Indices inside the shard sampled with the uniforms u (the library's sampler)."""
        return self.st.measure(np.asarray(u, np.float64).reshape(1, -1))[0]


def _is_diagonal(U: np.ndarray) -> bool:
    return not np.any(U - np.diag(np.diag(U)))


class ShardedState:
    """A 2^n register over 2^nglobal shards (see the module docstring).

    nqubits, nglobal : n and g (shards of L = n - g qubits, L >= 1)
    dtype            : torch.complex64 or torch.complex128
    group            : torch.distributed process group, or None for the default
                       group when one is initialised (else every shard is local)
    backend          : callable (L, dtype) -> shard; default LibShard (CUDA)
    """

    def __init__(self, nqubits: int, nglobal: int, dtype=torch.complex128, group=None, backend=None):
        import torch.distributed as dist
        self.n, self.g = int(nqubits), int(nglobal)
        self.L = self.n - self.g
        if self.g < 0 or self.L < 1:
            raise ValueError("need 0 <= nglobal < nqubits")
        self.nshards = 1 << self.g
        if dist.is_available() and dist.is_initialized():
            self.group = group
            self.world = dist.get_world_size(group)
            self.rank = dist.get_rank(group)
        else:
            self.group, self.world, self.rank = None, 1, 0
        if self.nshards % self.world:
            raise ValueError(f"{self.nshards} shards do not split over {self.world} ranks")
        self.per_rank = self.nshards // self.world
        self.owned = list(range(self.rank * self.per_rank, (self.rank + 1) * self.per_rank))
        self.dtype = dtype
        self._make = backend if backend is not None else (lambda L, dt: LibShard(L, dt))
        self.pos = list(range(self.n))   # logical qubit -> physical bit
        self.who = list(range(self.n))   # physical bit -> logical qubit
        self.vecs = {"psi": [self._make(self.L, dtype) for _ in self.owned]}
        self.exchanges = 0
        self.reset()

    # ------------------------------------------------------------------ bookkeeping
    def _vector(self, name: str, dtype=None):
        if name not in self.vecs:
            self.vecs[name] = [self._make(self.L, dtype or self.dtype) for _ in self.owned]
        return self.vecs[name]

    def _drop(self, name: str):
        self.vecs.pop(name, None)

    def _rank_of(self, shard: int) -> int:
        import torch.distributed as dist
        r = shard // self.per_rank
        return dist.get_global_rank(self.group, r) if self.group is not None else r

    def _phys(self, x: int) -> int:
        """Physical index of logical basis index x under the current map."""
        p = 0
        for q in range(self.n):
            if (x >> q) & 1:
                p |= 1 << self.pos[q]
        return p

    def reset(self, x: int = 0):
        """|x> (logical basis index) on psi; other vectors are dropped."""
        for name in list(self.vecs):
            if name != "psi":
                self._drop(name)
        p = self._phys(int(x))
        s_x, loc = p >> self.L, p & ((1 << self.L) - 1)
        for s, v in zip(self.owned, self.vecs["psi"]):
            if s == s_x:
                v.reset(loc)
            else:
                v.zero()
        return self

    def _sum(self, values: np.ndarray) -> np.ndarray:
        """Sum of a float64 vector over the ranks of the group."""
        import torch.distributed as dist
        v = np.ascontiguousarray(values, dtype=np.float64)
        if self.world == 1:
            return v
        dev = torch.device("cuda") if dist.get_backend(self.group) == "nccl" else torch.device("cpu")
        t = torch.as_tensor(v, device=dev).clone()
        dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()

    # ------------------------------------------------------------------ exchange
    def _exchange(self, l: int, j: int):
        """Swap physical local bit l with global bit j (physical L + j) in every vector."""
        import torch.distributed as dist
        L = self.L
        run = 2 << l                      # one run of 2^l amplitudes, in reals
        nrun = 1 << (L - 1 - l)
        for vecs in self.vecs.values():
            flats = {s: v.flat() for s, v in zip(self.owned, vecs)}
            tmp = None
            ops, back = [], []
            for idx, s in enumerate(self.owned):
                p = s ^ (1 << j)
                b = (s >> j) & 1
                x = flats[s]
                if p in flats:                       # partner in this process
                    if b == 1:
                        continue                      # handled from the b = 0 side
                    y = flats[p]
                    for a in range(nrun):
                        xs = x[(2 * a + 1) * run:(2 * a + 2) * run]   # s: bit l = 1
                        ys = y[(2 * a) * run:(2 * a + 1) * run]       # p: bit l = 0
                        t = xs.clone()
                        xs.copy_(ys)
                        ys.copy_(t)
                    continue
                if tmp is None:
                    tmp = torch.empty(nrun * run * len(self.owned), dtype=x.dtype, device=x.device)
                peer = self._rank_of(p)
                for a in range(nrun):
                    lo = (2 * a + (1 - b)) * run       # runs with bit l = 1 - b
                    rv = tmp[(idx * nrun + a) * run:(idx * nrun + a + 1) * run]
                    ops.append(dist.P2POp(dist.isend, x[lo:lo + run], peer, self.group, tag=idx * nrun + a))
                    ops.append(dist.P2POp(dist.irecv, rv, peer, self.group, tag=idx * nrun + a))
                    back.append((x[lo:lo + run], rv))
            if ops:
                for w in dist.batch_isend_irecv(ops):
                    w.wait()
                for dst, src in back:
                    dst.copy_(src)
        ql, qg = self.who[l], self.who[L + j]
        self.who[l], self.who[L + j] = qg, ql
        self.pos[qg], self.pos[ql] = l, L + j
        self.exchanges += 1

    def _localize(self, qubits):
        """Brings every logical qubit of `qubits` to a local physical bit."""
        need = [q for q in qubits if self.pos[q] >= self.L]
        if len(set(qubits)) > self.L:
            raise ValueError(f"{len(set(qubits))} qubits cannot all be local with {self.L} local bits")
        for q in need:
            keep = set(qubits)
            for l in range(self.L - 1, -1, -1):
                if self.who[l] not in keep:
                    break
            else:
                raise ValueError("no local bit to give up")
            self._exchange(l, self.pos[q] - self.L)

    # ------------------------------------------------------------------ gates
    def _restrict(self, s: int, ctrl_locs, ctrl_vals):
        """(applies, local control positions, values) of shard s."""
        lc, lv = [], []
        for c, v in zip(ctrl_locs, ctrl_vals):
            p = self.pos[c]
            if p >= self.L:
                if ((s >> (p - self.L)) & 1) != int(v):
                    return False, None, None
            else:
                lc.append(p)
                lv.append(int(v))
        return True, lc, lv

    def apply_matrix(self, U, locs, ctrl_locs=(), ctrl_vals=None, vectors=("psi",)):
        """instruct!(reg, U, locs, ctrl_locs, ctrl_vals) on the named vectors (logical qubits)."""
        locs = [int(q) for q in locs]
        ctrl_locs = [int(q) for q in ctrl_locs]
        ctrl_vals = [1] * len(ctrl_locs) if ctrl_vals is None else [int(v) for v in ctrl_vals]
        k = len(locs)
        U = np.asarray(U, dtype=np.complex128).reshape(1 << k, 1 << k)
        diag = _is_diagonal(U)
        if not diag:
            self._localize(locs)
        d = np.diag(U)
        for name in vectors:
            for s, v in zip(self.owned, self._vector(name)):
                ok, lc, lv = self._restrict(s, ctrl_locs, ctrl_vals)
                if not ok:
                    continue
                if not diag:
                    v.apply_matrix(U, [self.pos[q] for q in locs], lc, lv)
                    continue
                gl = [(j, self.pos[q] - self.L) for j, q in enumerate(locs) if self.pos[q] >= self.L]
                ll = [j for j, q in enumerate(locs) if self.pos[q] < self.L]
                dl = np.zeros(1 << len(ll), np.complex128)
                for m in range(1 << k):
                    if all(((m >> j) & 1) == ((s >> gb) & 1) for j, gb in gl):
                        dl[sum(((m >> j) & 1) << t for t, j in enumerate(ll))] = d[m]
                if ll:
                    if np.any(dl != 1):
                        v.apply_matrix(np.diag(dl), [self.pos[locs[j]] for j in ll], lc, lv)
                elif dl[0] != 1:
                    free = next(p for p in range(self.L) if p not in lc)
                    v.apply_matrix(np.diag([dl[0], dl[0]]), [free], lc, lv)
        return self

    def apply(self, g, params=None, vectors=("psi",)):
        """One gate record, matrix from the library's gate definitions."""
        U = qsim.gate_desc_matrices(g, params)
        return self.apply_matrix(U, g.locs, g.ctrl_locs, g.ctrl_vals, vectors)

    def apply_circuit(self, circuit: "qsim.Circuit", params=None):
        """apply!(reg, chain): the circuit's gates in order."""
        for i, g in enumerate(circuit.gates):
            U = circuit.gate_matrices(i, params)
            self.apply_matrix(U, g.locs, g.ctrl_locs, g.ctrl_vals)
        return self

    # ------------------------------------------------------------------ observables
    def _local_terms(self, s: int, terms):
        """Pauli terms evaluable on shard s: physical local positions, signed coefficients."""
        out = []
        for coeff, ops in terms:
            sign = 1.0
            local = []
            for q, P in ops:
                p = self.pos[q]
                if p >= self.L:
                    if P != "Z":
                        raise AssertionError("X/Y on a global qubit")
                    if (s >> (p - self.L)) & 1:
                        sign = -sign
                else:
                    local.append((p, P))
            out.append((sign * float(coeff), tuple(local)))
        return out

    def _batches(self, terms):
        """Runs of consecutive terms whose X/Y qubits are all local after one localisation."""
        batch = []
        for term in terms:
            xy = [q for q, P in term[1] if P != "Z"]
            if any(self.pos[q] >= self.L for q in xy):
                if batch:
                    yield batch
                    batch = []
                self._localize(xy)
            batch.append(term)
        if batch:
            yield batch

    def expect(self, terms) -> float:
        """<psi|O|psi> for O = sum coeff P (terms as qsim.Observable takes them)."""
        total = 0.0
        for batch in self._batches(list(terms)):
            for s, v in zip(self.owned, self.vecs["psi"]):
                total += v.expect(self._local_terms(s, batch))
        return float(self._sum(np.array([total]))[0])

    def _apply_observable(self, terms, src: str, dst: str, tmp: str, dtype=None):
        """dst <- O src, one Pauli string at a time through tmp (the library's Pauli
        gates on local bits, a global Z read as the shard's sign)."""
        for v in self._vector(dst, dtype):
            v.zero()
        self._vector(tmp, dtype)
        for batch in self._batches(list(terms)):
            for coeff, ops in batch:
                for s, vt, vs, vd in zip(self.owned, self.vecs[tmp], self.vecs[src], self.vecs[dst]):
                    vt.copy_from(vs)
                    sign = 1.0
                    local = []
                    for q, P in ops:
                        p = self.pos[q]
                        if p >= self.L:
                            sign = -sign if (s >> (p - self.L)) & 1 else sign
                        else:
                            local.append((p, P))
                    for p, P in local:
                        vt.apply_pauli(p, P)
                    vd.axpy(-float(coeff) if sign < 0 else float(coeff), vt)

    # ------------------------------------------------------------------ gradient
    def backward(self, circuit: "qsim.Circuit", params, terms):
        """expect'(O, reg => circuit): psi holds the circuit's output state; returns
        (loss, gradient).  psi is uncomputed to the circuit's input state (for a
        complex64 register, rounded back from the FP64 walk)."""
        params = np.asarray(params, dtype=np.float64)
        loss = self.expect(terms)
        wide = torch.complex128
        work = "psi"
        if self.dtype != wide:
            work = "psiw"
            for vw, vs in zip(self._vector(work, wide), self.vecs["psi"]):
                vw.copy_from(vs)
        self._apply_observable(terms, work, "lam", "tmp", dtype=wide)
        self._drop("tmp")
        grad = self.vecs[work][0].new_grad(circuit.nparams)
        for i in range(len(circuit.gates) - 1, -1, -1):
            g = circuit.gates[i]
            if g.param is not None and g.name != "MATRIX":
                self._localize(list(g.locs))
                for s, vp, vl in zip(self.owned, self.vecs[work], self.vecs["lam"]):
                    ok, lc, lv = self._restrict(s, g.ctrl_locs, g.ctrl_vals)
                    if not ok:
                        continue  # identity on this shard, and its control projector is zero here
                    local = dataclasses.replace(g, locs=tuple(self.pos[q] for q in g.locs),
                                                ctrl_locs=tuple(lc), ctrl_vals=tuple(lv))
                    vp.adjoint_step(vl, local, params, grad)
            else:
                Ud = qsim.gate_desc_matrices(g, params, dagger=True)
                self.apply_matrix(Ud, g.locs, g.ctrl_locs, g.ctrl_vals, vectors=(work, "lam"))
        grad = self._sum(self.vecs[work][0].grad_host(grad))
        if work != "psi":
            for vs, vw in zip(self.vecs["psi"], self.vecs[work]):
                vs.copy_from(vw)
            self._drop(work)
        self._drop("lam")
        return loss, grad[:circuit.nparams]

    # ------------------------------------------------------------------ measurement
    def _logical(self, phys: np.ndarray) -> np.ndarray:
        x = np.zeros_like(phys)
        for q in range(self.n):
            x |= ((phys >> self.pos[q]) & 1) << q
        return x

    def measure(self, u) -> np.ndarray:
        """Logical basis indices sampled from |psi|^2 with the uniforms u in [0, 1),
        one per shot; the state is unchanged.  Shard s is drawn with probability
        P_s / T (t = u T walked over the left-fold prefixes of the shard weights
        P_s = <psi_s|psi_s>, FP64), the index inside it by the shard's sampler with
        u' = (t - prefix) / P_s; with one shard, the register's sampler with u.
        Every rank returns all shots."""
        u = np.ascontiguousarray(np.ravel(u), dtype=np.float64)
        if not np.all((u >= 0.0) & (u < 1.0)):
            raise ValueError("uniforms must lie in [0, 1)")
        psi = self.vecs["psi"]
        if self.nshards == 1:
            return self._logical(np.asarray(psi[0].measure(u), np.int64))
        w = np.zeros(self.nshards)
        for s, v in zip(self.owned, psi):
            w[s] = v.inner(v).real
        w = self._sum(w)
        pick, sub = qsim.sample_shards(w, u)
        phys = np.zeros(len(u), np.float64)
        for s, v in zip(self.owned, psi):
            m = pick == s
            if m.any():
                phys[m] = (s << self.L) | np.asarray(v.measure(sub[m]), np.int64)
        return self._logical(self._sum(phys).astype(np.int64))

    # ------------------------------------------------------------------ host views (small n)
    def _perm(self) -> np.ndarray:
        """perm[x] = physical index of logical index x under the current map."""
        idx = np.arange(1 << self.n, dtype=np.int64)
        perm = np.zeros_like(idx)
        for q in range(self.n):
            perm |= ((idx >> q) & 1) << self.pos[q]
        return perm

    def upload(self, amps):
        """psi <- a whole register given in logical order (host memory; every rank
        passes the same array and keeps its own shards)."""
        amps = np.asarray(amps, dtype=np.complex128).ravel()
        if amps.size != 1 << self.n:
            raise ValueError("amplitude count does not match the register")
        for name in list(self.vecs):
            if name != "psi":
                self._drop(name)
        phys = np.empty_like(amps)
        phys[self._perm()] = amps
        for s, v in zip(self.owned, self.vecs["psi"]):
            v.upload(phys[s << self.L:(s + 1) << self.L])
        return self

    def local_shards(self, name: str = "psi") -> dict:
        return {s: v.numpy() for s, v in zip(self.owned, self._vector(name))}

    def gather(self, name: str = "psi") -> np.ndarray:
        """The whole register in logical order on every rank (host memory; for small n)."""
        import torch.distributed as dist
        mine = np.concatenate([self.local_shards(name)[s] for s in self.owned]).astype(np.complex128)
        if self.world > 1:
            dev = torch.device("cuda") if dist.get_backend(self.group) == "nccl" else torch.device("cpu")
            t = torch.view_as_real(torch.as_tensor(mine)).contiguous().to(dev)
            parts = [torch.empty_like(t) for _ in range(self.world)]
            dist.all_gather(parts, t, group=self.group)
            phys = np.concatenate([torch.view_as_complex(p.cpu()).numpy() for p in parts])
        else:
            phys = mine
        return phys[self._perm()]
