"""Python binding of the GB300 state-vector library (include/qsim.h).

PyTorch provides device memory and streams only; every step of the simulation
runs in libqsim.so's CUDA kernels.  Gate lists use the ``workloads.Gate``
record (name, locs, ctrl_locs, ctrl_vals, param, theta, paulis, matrix); this
module only marshals them into ``qs_gate_desc`` arrays.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N

_TORCH_DTYPE = {N.QS_C64: torch.complex64, N.QS_C128: torch.complex128}
_NP_DTYPE = {N.QS_C64: np.complex64, N.QS_C128: np.complex128}


def _dtype_code(dtype) -> int:
    if dtype in (N.QS_C64, torch.complex64, np.complex64, "c64", "complex64"):
        return N.QS_C64
    if dtype in (N.QS_C128, torch.complex128, np.complex128, "c128", "complex128"):
        return N.QS_C128
    raise ValueError(f"unsupported dtype {dtype}")


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class State:
    """A register or a batch of registers in device memory owned by a torch tensor
    (Sec. "Quantum Registers", Sec. "Batched Quantum Registers")."""

    def __init__(self, nqubits, dtype=torch.complex64, nbatch: int = 1, device="cuda", stream=None):
        L = N.lib()
        self.dtype_code = _dtype_code(dtype)
        if isinstance(nqubits, (list, tuple, np.ndarray)):
            counts = [int(x) for x in nqubits]
        else:
            counts = [int(nqubits)] * int(nbatch)
        self.counts = counts
        self.nreg = len(counts)
        self.uniform = len(set(counts)) == 1
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("State lives on a CUDA device")
        total = sum(1 << c for c in counts)
        self.buffer = torch.empty(total, dtype=_TORCH_DTYPE[self.dtype_code], device=self.device)
        self.stream = stream
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            N.check(L.qs_batch_create(self.nreg, N.i32(counts), self.dtype_code,
                                      ctypes.c_void_p(self.buffer.data_ptr()), _stream_ptr(stream),
                                      ctypes.byref(h)))
        self.handle = h
        self.offsets = np.cumsum([0] + [1 << c for c in counts])

    # -- lifetime -----------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            N.lib().qs_state_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nqubits(self) -> int:
        if not self.uniform:
            raise ValueError("uneven batch: use .counts")
        return self.counts[0]

    def sync_stream(self, stream=None):
        N.check(N.lib().qs_state_set_stream(self.handle, _stream_ptr(stream)))
        self.stream = stream

    def sync(self):
        """Waits for the state's stream; raises if a tensor-core wait gave up."""
        N.check(N.lib().qs_state_sync(self.handle))

    # -- data -----------------------------------------------------------------
    def register(self, r: int) -> torch.Tensor:
        return self.buffer[int(self.offsets[r]):int(self.offsets[r + 1])]

    def tensor(self) -> torch.Tensor:
        """[nbatch, 2^n] view (uniform batches) of the amplitudes."""
        return self.buffer.view(self.nreg, -1)

    def reset(self, basis=None):
        if basis is None:
            N.check(N.lib().qs_state_reset(self.handle, None))
        else:
            b = np.ascontiguousarray(np.broadcast_to(np.asarray(basis, dtype=np.uint64), (self.nreg,)))
            N.check(N.lib().qs_state_reset(self.handle, b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))
        return self

    def upload(self, amps: np.ndarray):
        a = np.ascontiguousarray(np.ravel(amps), dtype=_NP_DTYPE[self.dtype_code])
        if a.size != int(self.offsets[-1]):
            raise ValueError("amplitude count does not match the state")
        N.check(N.lib().qs_state_upload(self.handle, a.ctypes.data))
        return self

    def numpy(self) -> np.ndarray:
        out = np.empty(int(self.offsets[-1]), dtype=_NP_DTYPE[self.dtype_code])
        N.check(N.lib().qs_state_download(self.handle, out.ctypes.data))
        return out

    # -- level-1 operations between states of the same shape -------------------
    def copy_from(self, src: "State"):
        """self <- src (stream-ordered on self's stream)."""
        N.check(N.lib().qs_state_copy(self.handle, src.handle))
        return self

    def inner(self, other: "State") -> np.ndarray:
        """<self_r|other_r> per register (FP64 sums), complex128 [nreg]."""
        out = np.zeros(2 * self.nreg)
        N.check(N.lib().qs_state_inner(self.handle, other.handle, N.dptr(out)))
        return out.view(np.complex128)

    def axpy(self, alpha, x: "State"):
        """self <- self + alpha x."""
        a = complex(alpha)
        N.check(N.lib().qs_state_axpy(self.handle, a.real, a.imag, x.handle))
        return self

    # -- instructions ---------------------------------------------------------
    def apply(self, g, params=None):
        """instruct! one gate record (workloads.Gate): Sec. "Instructions on Quantum
        Registers", the general multi-control instruction of Sec. "Performance"."""
        cl = N.i32(g.ctrl_locs)
        cv = N.i32(g.ctrl_vals)
        locs = N.i32(g.locs)
        if g.name == "MATRIX":
            m = np.ascontiguousarray(g.matrix, dtype=np.complex128).view(np.float64)
            N.check(N.lib().qs_apply_gate(self.handle, N.dptr(m), len(g.locs), locs,
                                          len(g.ctrl_locs), cl, cv))
        else:
            theta = 0.0
            if g.param is not None:
                theta = float(params[g.param])
            elif g.theta is not None:
                theta = float(g.theta)
            paulis = N.i32([N.PAULI_CODE[p] for p in g.paulis] if g.paulis else [])
            N.check(N.lib().qs_apply_named(self.handle, N.GATE_KIND[g.name], len(g.locs), locs, paulis,
                                           len(g.ctrl_locs), cl, cv, theta))
        return self

    def apply_matrix(self, U, locs, ctrl_locs=(), ctrl_vals=()):
        """instruct!(reg, U, locs, ctrl_locs, ctrl_vals) with a dense 2^k x 2^k matrix."""
        m = np.ascontiguousarray(U, dtype=np.complex128).view(np.float64)
        N.check(N.lib().qs_apply_gate(self.handle, N.dptr(m), len(locs), N.i32(locs), len(ctrl_locs),
                                      N.i32(ctrl_locs), N.i32(ctrl_vals or [1] * len(ctrl_locs))))
        return self

    def apply_circuit(self, circuit: "Circuit", params=None, per_register=False, fused=True, tiles=False,
                      tile_qubits=0, blocks=0, flags=None, precise=False):
        """apply!(reg, chain) (Sec. "Representing Quantum Circuits").  fused=False: one launch per gate; tiles=True: force the
        tile engine (fused passes over 2^tile_qubits-amplitude tiles); blocks=k: fuse
        the gates into blocks of at most k qubits; precise=True: complex64 gates (or blocks) with
        compensated matrices, each output rounded once (QS_APPLY_PRECISE); flags: raw qs_apply_circuit flags
        (e.g. from autotune), overriding the others."""
        p = _params_array(params, circuit.nparams * (self.nreg if per_register else 1))
        if flags is None:
            flags = (N.QS_APPLY_PER_REGISTER if per_register else 0) | (0 if fused else N.QS_APPLY_UNFUSED)
            flags |= N.QS_APPLY_PRECISE if precise else 0
            flags |= (N.QS_APPLY_TILES if tiles else 0) | (int(tile_qubits) << 8)
            if blocks:
                flags |= N.QS_APPLY_BLOCKS | (int(blocks) << 16)
        N.check(N.lib().qs_apply_circuit(self.handle, circuit.handle, N.dptr(p), int(flags)))
        return self

    def expect(self, obs: "Observable") -> np.ndarray:
        """expect(O, reg) per register (Sec. "Forward Mode"), FP64 sums."""
        out = np.zeros(self.nreg)
        N.check(N.lib().qs_expect(self.handle, obs.handle, N.dptr(out)))
        return out

    def measure(self, u, collapse=False) -> np.ndarray:
        """measure / measure! (Sec. "Instructions on Quantum Registers"): basis indices
        sampled with the given uniforms [nreg][nshots] in [0, 1) under the sampling
        contract of qsim.h; collapse=True projects onto the single sampled state."""
        u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(self.nreg, -1))
        out = np.zeros(u.shape, dtype=np.int64)
        N.check(N.lib().qs_measure(self.handle, N.dptr(u), u.shape[1],
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 1 if collapse else 0))
        return out

    def measure_seeded(self, seed: int, nshots: int, collapse=False) -> np.ndarray:
        """measure with the uniforms drawn on the device from ``seed`` (SplitMix64, see
        qs_measure_seeded in qsim.h): [nreg][nshots] basis indices fixed by the seed."""
        out = np.zeros((self.nreg, int(nshots)), dtype=np.int64)
        N.check(N.lib().qs_measure_seeded(self.handle, ctypes.c_uint64(int(seed) & ((1 << 64) - 1)), int(nshots),
                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 1 if collapse else 0))
        return out


def _params_array(params, count):
    if count == 0:
        return np.zeros(1)
    p = np.ascontiguousarray(np.ravel(np.asarray(params, dtype=np.float64)))
    if p.size != count:
        raise ValueError(f"expected {count} parameters, got {p.size}")
    return p


def _fill_desc(d, g, off: int, pool: list) -> int:
    """Marshals one workloads.Gate into a qs_gate_desc; MATRIX entries go to `pool`
    at complex offset `off`.  Returns the next free offset."""
    d.kind = N.GATE_KIND[g.name]
    d.nlocs = len(g.locs)
    for j, l in enumerate(g.locs):
        d.locs[j] = l
    if g.paulis:
        for j, p in enumerate(g.paulis):
            d.paulis[j] = N.PAULI_CODE[p]
    d.param = -1 if g.param is None else int(g.param)
    d.theta = 0.0 if g.theta is None else float(g.theta)
    cm = cv = 0
    for l, v in zip(g.ctrl_locs, g.ctrl_vals):
        cm |= 1 << l
        if v:
            cv |= 1 << l
    d.ctrl_mask, d.ctrl_vals = cm, cv
    if g.name == "MATRIX":
        m = np.ascontiguousarray(g.matrix, dtype=np.complex128).ravel()
        d.mat_offset = off
        pool.append(m)
        off += m.size
    return off


def gate_record(g):
    """(qs_gate_desc, matrix pool as interleaved doubles) of one gate record."""
    d = N.GateDesc()
    pool = []
    _fill_desc(d, g, 0, pool)
    mats = np.concatenate(pool) if pool else np.zeros(1, np.complex128)
    return d, np.ascontiguousarray(mats).view(np.float64)


def gate_desc_matrices(g, params=None, dagger: bool = False, generator: bool = False):
    """U (or U^dagger) of one gate record from the library's gate definitions, and with
    generator=True also (H, c) with U = exp(-i theta c H) (qs_gate_desc_matrices)."""
    d, mats = gate_record(g)
    D = 1 << len(g.locs)
    p = np.ascontiguousarray(np.zeros(1) if params is None or len(params) == 0 else params, dtype=np.float64)
    U = np.zeros(2 * D * D)
    G = np.zeros(2 * D * D) if generator else None
    cf = ctypes.c_double()
    N.check(N.lib().qs_gate_desc_matrices(ctypes.byref(d), N.dptr(mats), N.dptr(p), 1 if dagger else 0, N.dptr(U),
                                          N.dptr(G) if generator else None,
                                          ctypes.byref(cf) if generator else None))
    U = U.view(np.complex128).reshape(D, D)
    if not generator:
        return U
    return U, G.view(np.complex128).reshape(D, D), cf.value


def adjoint_step(psi: "State", lam: "State", g, params, dev_grad: torch.Tensor):
    """One gate of the reversible adjoint walk on complex128 registers psi and lam
    (qs_adjoint_step): dev_grad[g.param] += 2 c Im<lam|P_ctrl H|psi> for a parameterised
    gate, then psi, lam <- U^dag psi, U^dag lam.  Asynchronous; dev_grad: float64 CUDA."""
    d, mats = gate_record(g)
    p = np.ascontiguousarray(np.zeros(1) if params is None or len(params) == 0 else params, dtype=np.float64)
    N.check(N.lib().qs_adjoint_step(psi.handle, lam.handle, ctypes.byref(d), N.dptr(mats), N.dptr(p),
                                    ctypes.c_void_p(dev_grad.data_ptr())))


def sample_shards(weights, u):
    """First level of a measurement over shards (qs_sample_shards): per uniform, the shard
    drawn from the shard weights and the uniform its own sampler takes."""
    w = np.ascontiguousarray(weights, dtype=np.float64)
    u = np.ascontiguousarray(np.ravel(u), dtype=np.float64)
    shard = np.zeros(len(u), np.int32)
    sub = np.zeros(len(u))
    N.check(N.lib().qs_sample_shards(len(w), N.dptr(w), len(u), N.dptr(u), shard.ctypes.data_as(N._PI32),
                                     N.dptr(sub)))
    return shard.astype(np.int64), sub


class Circuit:
    """Immutable flat gate list (qs_circuit): the put / control / chain blocks of
    Sec. "Representing Quantum Circuits" flattened into gate records."""

    def __init__(self, gates, nqubits: int, nparams: int | None = None):
        L = N.lib()
        if nparams is None:
            nparams = 1 + max([g.param for g in gates if g.param is not None], default=-1)
        arr = (N.GateDesc * max(1, len(gates)))()
        pool = []
        off = 0
        for i, g in enumerate(gates):
            off = _fill_desc(arr[i], g, off, pool)
        mats = np.concatenate(pool) if pool else np.zeros(1, np.complex128)
        mv = mats.view(np.float64)
        h = ctypes.c_void_p()
        N.check(L.qs_circuit_create(int(nqubits), arr, len(gates), N.dptr(mv), off, int(nparams), ctypes.byref(h)))
        self.handle = h
        self.nqubits = int(nqubits)
        self.nparams = int(nparams)
        self.ngates = len(gates)
        self.gates = list(gates)

    def gate_matrices(self, index: int, params=None, generator: bool = False):
        """Host-side matrices of gate `index`: U at `params` (2^k x 2^k complex128) and,
        with generator=True, (H, c) with U = exp(-i theta c H)."""
        g = self.gates[index]
        D = 1 << len(g.locs)
        p = _params_array(params, self.nparams) if self.nparams else np.zeros(1)
        U = np.zeros(2 * D * D)
        G = np.zeros(2 * D * D) if generator else None
        cf = ctypes.c_double()
        N.check(N.lib().qs_circuit_gate_matrices(self.handle, int(index), N.dptr(p), None, N.dptr(U),
                                                 N.dptr(G) if generator else None,
                                                 ctypes.byref(cf) if generator else None))
        U = U.view(np.complex128).reshape(D, D)
        if not generator:
            return U
        return U, G.view(np.complex128).reshape(D, D), cf.value

    def checkpoint_count(self, every: int) -> int:
        c = ctypes.c_int()
        N.check(N.lib().qs_checkpoint_count(self.handle, int(every), ctypes.byref(c)))
        return c.value

    def __del__(self):
        try:
            if self.handle.value:
                N.lib().qs_circuit_destroy(self.handle)
                self.handle = ctypes.c_void_p()
        except Exception:
            pass


class Observable:
    """sum_t coeff_t P_t from terms [(coeff, ((loc, 'X'|'Y'|'Z'), ...)), ...] (the
    Hamiltonians of Sec. "Forward Mode" and Listing "Heisenberg Hamiltonian")."""

    def __init__(self, terms):
        arr = (N.PauliTerm * max(1, len(terms)))()
        for i, (c, ops) in enumerate(terms):
            x = z = 0
            for l, p in ops:
                if p in ("X", "Y"):
                    x |= 1 << int(l)
                if p in ("Z", "Y"):
                    z |= 1 << int(l)
            arr[i].coeff, arr[i].x_mask, arr[i].z_mask = float(c), x, z
        h = ctypes.c_void_p()
        N.check(N.lib().qs_observable_create(arr, len(terms), ctypes.byref(h)))
        self.handle = h
        self.terms = list(terms)

    def __del__(self):
        try:
            if self.handle.value:
                N.lib().qs_observable_destroy(self.handle)
                self.handle = ctypes.c_void_p()
        except Exception:
            pass


def backward_work(nqubits: int, device="cuda") -> torch.Tensor:
    b = ctypes.c_size_t()
    N.check(N.lib().qs_backward_work_bytes(int(nqubits), ctypes.byref(b)))
    return torch.empty(b.value, dtype=torch.uint8, device=device)


def checkpoint_buffer(state: State, circuit: Circuit, every: int) -> torch.Tensor | None:
    cnt = circuit.checkpoint_count(every)
    if every <= 0 or cnt == 0:
        return None
    return torch.empty((cnt, state.buffer.numel()), dtype=state.buffer.dtype, device=state.buffer.device)


def apply_circuit_ckpt(state: State, circuit: Circuit, params, every: int, ckpts: torch.Tensor | None):
    p = _params_array(params, circuit.nparams)
    ptr = ctypes.c_void_p(ckpts.data_ptr()) if ckpts is not None else None
    N.check(N.lib().qs_apply_circuit_ckpt(state.handle, circuit.handle, N.dptr(p), int(every), ptr))
    return state


def backward(state: State, circuit: Circuit, params, obs: Observable, ckpt_every: int = 0,
             ckpts: torch.Tensor | None = None, work: torch.Tensor | None = None):
    """expect'(O, reg => circuit): (loss, grad) from the circuit's output state (left
    unchanged), by the reversible adjoint of Sec. "Reverse Mode" (Eq. apply-back)."""
    p = _params_array(params, circuit.nparams)
    if work is None:
        work = backward_work(state.nqubits, state.device)
    grad = np.zeros(max(1, circuit.nparams))
    loss = np.zeros(1)
    ck = ctypes.c_void_p(ckpts.data_ptr()) if ckpts is not None else None
    N.check(N.lib().qs_backward(state.handle, circuit.handle, N.dptr(p), obs.handle, int(ckpt_every), ck,
                                ctypes.c_void_p(work.data_ptr()), N.dptr(grad), N.dptr(loss)))
    return float(loss[0]), grad[:circuit.nparams]


class BatchProgram:
    """Per-register circuits and diagonal observables of a batch of uneven registers,
    scheduled once into fused tile passes (qs_batch_program).  phase_qubits: the fusion
    width (qubits whose gates a phase applies in registers, 2..4; 0 = 4, 3 when precise); precise: the
    compensated forward and double-float uncompute of qs_batch_program_create_ex."""

    def __init__(self, circuits, observables, tile_qubits: int = 0, phase_qubits: int = 0, precise: bool = False):
        L = N.lib()
        nreg = len(circuits)
        if len(observables) != nreg:
            raise ValueError("one observable per register")
        ch = (ctypes.c_void_p * nreg)(*[c.handle.value for c in circuits])
        oh = (ctypes.c_void_p * nreg)(*[o.handle.value for o in observables])
        h = ctypes.c_void_p()
        N.check(L.qs_batch_program_create_ex(nreg, ctypes.cast(ch, ctypes.POINTER(ctypes.c_void_p)),
                                             ctypes.cast(oh, ctypes.POINTER(ctypes.c_void_p)), int(tile_qubits),
                                             int(phase_qubits), N.QS_BATCH_PRECISE if precise else 0,
                                             ctypes.byref(h)))
        self.handle = h
        t, ph, fl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        N.check(L.qs_batch_program_shape(h, ctypes.byref(t), ctypes.byref(ph), ctypes.byref(fl)))
        self.tile_qubits, self.phase_qubits, self.precise = t.value, ph.value, bool(fl.value & N.QS_BATCH_PRECISE)
        self.nreg = nreg
        self.counts = [c.nqubits for c in circuits]
        tot = ctypes.c_int64()
        po = np.zeros(nreg + 1, np.int64)
        ao = np.zeros(nreg + 1, np.int64)
        N.check(L.qs_batch_program_info(h, None, ctypes.byref(tot), po.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                        ao.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        self.nparams = int(tot.value)
        self.param_offsets = po
        self.amp_offsets = ao
        self._keep = (circuits, observables)

    def run(self, state: State, params: torch.Tensor, grad: bool = True, reset: bool = True,
            loss: torch.Tensor | None = None, grad_out: torch.Tensor | None = None):
        """One persistent launch: forward (+ backward).  params: flat float64 CUDA tensor."""
        if params.dtype != torch.float64 or not params.is_cuda or params.numel() != self.nparams:
            raise ValueError("params must be a float64 CUDA tensor of nparams entries")
        params = params.contiguous()
        if loss is None:
            loss = torch.empty(self.nreg, dtype=torch.float64, device=params.device)
        if grad and grad_out is None:
            grad_out = torch.empty(self.nparams, dtype=torch.float64, device=params.device)
        flags = (N.QS_BATCH_RESET if reset else 0) | (N.QS_BATCH_GRAD if grad else 0)
        N.check(N.lib().qs_batch_run(state.handle, self.handle, ctypes.c_void_p(params.data_ptr()),
                                     ctypes.c_void_p(loss.data_ptr()),
                                     ctypes.c_void_p(grad_out.data_ptr() if grad else 0), flags))
        return loss, grad_out

    def __del__(self):
        try:
            if self.handle.value:
                N.lib().qs_batch_program_destroy(self.handle)
                self.handle = ctypes.c_void_p()
        except Exception:
            pass


def backward_tiled(state: State, circuit: Circuit, params, obs: Observable, tile_qubits: int = 0,
                   work: torch.Tensor | None = None):
    """expect' for a large complex64 register on the tile engine (FP32 uncompute,
    FP64 gradient accumulation): (loss, grad); the state is left unchanged."""
    p = _params_array(params, circuit.nparams)
    if work is None:
        b = ctypes.c_size_t()
        N.check(N.lib().qs_backward_tiled_work_bytes(state.nqubits, ctypes.byref(b)))
        work = torch.empty(b.value, dtype=torch.uint8, device=state.device)
    grad = np.zeros(max(1, circuit.nparams))
    loss = np.zeros(1)
    N.check(N.lib().qs_backward_tiled(state.handle, circuit.handle, N.dptr(p), obs.handle, int(tile_qubits),
                                      ctypes.c_void_p(work.data_ptr()), N.dptr(grad), N.dptr(loss)))
    return float(loss[0]), grad[:circuit.nparams]


def schedule_info(circuit: Circuit, tile_qubits: int = 0):
    """(passes, phases) of the circuit's tile-engine schedule (gates reordered only
    past gates on disjoint qubits, Sec. "Representing Quantum Circuits")."""
    p, f = ctypes.c_int(), ctypes.c_int()
    N.check(N.lib().qs_circuit_schedule_info(circuit.handle, int(tile_qubits), ctypes.byref(p), ctypes.byref(f)))
    return p.value, f.value


def tile_order(circuit: Circuit, tile_qubits: int = 0):
    """(order, pass) of the tile engine's schedule, host only: order[i] indexes the
    circuit's gate list with every SWAP rewritten as three controlled X gates."""
    L = N.lib()
    cnt = ctypes.c_int()
    N.check(L.qs_circuit_tile_order(circuit.handle, int(tile_qubits), ctypes.byref(cnt), None, None))
    order = np.zeros(max(1, cnt.value), np.int32)
    passes = np.zeros(max(1, cnt.value), np.int32)
    P32 = ctypes.POINTER(ctypes.c_int32)
    N.check(L.qs_circuit_tile_order(circuit.handle, int(tile_qubits), ctypes.byref(cnt),
                                    order.ctypes.data_as(P32), passes.ctypes.data_as(P32)))
    return order[:cnt.value], passes[:cnt.value]


def set_tensor_cores(mode) -> None:
    """Kernel for dense 4- and 5-qubit complex64 gates: True or 2 = always the tensor
    cores, False or 0 = the CUDA cores, 1 = per target placement (default)."""
    m = 2 if mode is True else (0 if mode is False else int(mode))
    N.check(N.lib().qs_set_option(N.QS_OPT_TENSOR_CORES, m))


def tensor_cores() -> int:
    v = ctypes.c_int(0)
    N.check(N.lib().qs_get_option(N.QS_OPT_TENSOR_CORES, ctypes.byref(v)))
    return v.value


def circuit_blocks(circuit: Circuit, params=None, kmax: int = 5, matrices: bool = True):
    """The k-qubit blocks of circuit (application order): list of (qubits, matrix or None);
    a block's matrix is the product of its gates (Sec. "Matrix Representation")."""
    L = N.lib()
    nb = ctypes.c_int(0)
    p = _params_array(params, circuit.nparams)
    N.check(L.qs_circuit_blocks(circuit.handle, N.dptr(p), int(kmax), ctypes.byref(nb), None, None, None))
    n = nb.value
    widths = np.zeros(n, dtype=np.int32)
    locs = np.zeros(n * N.QS_MAXK, dtype=np.int32)
    stride = 1 << (2 * N.QS_MAXK)
    mats = np.zeros(n * stride, dtype=np.complex128) if matrices else None
    N.check(L.qs_circuit_blocks(circuit.handle, N.dptr(p), int(kmax), ctypes.byref(nb),
                                widths.ctypes.data_as(N._PI32), locs.ctypes.data_as(N._PI32),
                                N.dptr(mats.view(np.float64)) if matrices else None))
    out = []
    for b in range(n):
        w = int(widths[b])
        q = tuple(int(x) for x in locs[b * N.QS_MAXK:b * N.QS_MAXK + w])
        m = None
        if matrices:
            d = 1 << w
            m = mats[b * stride:b * stride + d * d].reshape(d, d).copy()
        out.append((q, m))
    return out


def autotune(state: State, circuit: Circuit, params=None, reps: int = 3):
    """Times the circuit under each fusion / tile candidate on this state (whose
    amplitudes are overwritten) and returns (best_flags, {flags: ms})."""
    L = N.lib()
    p = _params_array(params, circuit.nparams)
    cap = 32
    best = ctypes.c_int(0)
    nc = ctypes.c_int(cap)
    cf = np.zeros(cap, dtype=np.int32)
    cm = np.zeros(cap, dtype=np.float64)
    N.check(L.qs_autotune_circuit(state.handle, circuit.handle, N.dptr(p), int(reps), ctypes.byref(best),
                                  ctypes.byref(nc), cf.ctypes.data_as(N._PI32), N.dptr(cm)))
    return best.value, {int(cf[i]): float(cm[i]) for i in range(min(nc.value, cap))}


def backward_blocks(state: State, circuit: Circuit, params, obs: Observable, kmax: int = 5, work=None):
    """Reversible gradient over k-qubit blocks: (loss, grad); the state is uncomputed to
    the circuit's input.  work: optional device buffer of one state."""
    L = N.lib()
    b = ctypes.c_size_t()
    N.check(L.qs_backward_blocks_work_bytes(int(circuit.nqubits), state.dtype_code, ctypes.byref(b)))
    if work is None:
        work = torch.empty(b.value, dtype=torch.uint8, device=state.buffer.device)
    p = _params_array(params, circuit.nparams)
    grad = np.zeros(max(1, circuit.nparams))
    loss = np.zeros(1)
    N.check(L.qs_backward_blocks(state.handle, circuit.handle, N.dptr(p), obs.handle, int(kmax),
                                 ctypes.c_void_p(work.data_ptr()), N.dptr(grad), N.dptr(loss)))
    return float(loss[0]), grad[:circuit.nparams]


def run_one_launch(state: State, circuit: Circuit, params=None, kmax: int = 4, obs: "Observable | None" = None,
                   grid_ctas: int = 0, out: torch.Tensor | None = None):
    """The whole circuit on one small register in a single cooperative launch
    (qs_run_circuit_one_launch), with <obs> (diagonal) evaluated in the same launch into
    `out` (a float64 CUDA tensor of one element, returned).  Asynchronous."""
    p = _params_array(params, circuit.nparams)
    if obs is not None and out is None:
        out = torch.empty(1, dtype=torch.float64, device=state.device)
    N.check(N.lib().qs_run_circuit_one_launch(state.handle, circuit.handle, N.dptr(p), int(kmax),
                                              obs.handle if obs is not None else None, int(grid_ctas),
                                              ctypes.c_void_p(out.data_ptr()) if out is not None else None))
    return out


class CapturedCircuit:
    """One apply of `circuit` (fixed parameters and flags) on `state`, recorded as a
    CUDA graph and replayed with a single launch: the remedy for launch-bound
    circuits on small registers.  The constructor applies the circuit once outside
    the capture (host plans, kernel attributes), so reset the state afterwards;
    `replay()` then applies it again in the state's memory."""

    def __init__(self, state: State, circuit: Circuit, params=None, **apply_kwargs):
        self.state = state
        self.stream = torch.cuda.Stream(device=state.device)
        prev = state.stream
        state.sync_stream(self.stream)
        try:
            with torch.cuda.stream(self.stream):
                state.apply_circuit(circuit, params, **apply_kwargs)
            self.stream.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=self.stream, capture_error_mode="thread_local"):
                state.apply_circuit(circuit, params, **apply_kwargs)
        finally:
            self.stream.synchronize()
            state.sync_stream(prev)

    def replay(self):
        self.graph.replay()
        return self


def observable_groups(obs: Observable) -> int:
    """Number of measurement-basis groups shot-based estimates use (uniform sets per register)."""
    g = ctypes.c_int(0)
    N.check(N.lib().qs_observable_groups(obs.handle, ctypes.byref(g)))
    return g.value


def shot_expect(state: State, obs: Observable, uniforms, work: torch.Tensor | None = None) -> np.ndarray:
    """Shot-based <O> per register; uniforms: [groups][nreg][nshots] in [0, 1)."""
    u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
    if u.ndim != 3 or u.shape[1] != state.nreg:
        raise ValueError("uniforms must be [groups][nreg][nshots]")
    if work is None:
        work = torch.empty_like(state.buffer)
    out = np.zeros(state.nreg)
    N.check(N.lib().qs_shot_expect(state.handle, obs.handle, N.dptr(u), int(u.shape[2]),
                                   ctypes.c_void_p(work.data_ptr()), N.dptr(out)))
    return out


def faithful_gradient(circuit: Circuit, params, obs: Observable, dtype=torch.complex128, nshots: int = 0,
                      uniforms=None, device="cuda") -> np.ndarray:
    """Eq. shiftrule gradient of <O> from |0...0> (exact, or from nshots samples per shifted
    circuit with uniforms [groups][2 nparams][nshots])."""
    P = circuit.nparams
    p = _params_array(params, P)
    code = _dtype_code(dtype)
    states = torch.empty((2 * P) << circuit.nqubits, dtype=_TORCH_DTYPE[code], device=device)
    work = torch.empty_like(states) if nshots > 0 else None
    u = None
    if nshots > 0:
        u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
        if u.shape[1:] != (2 * P, nshots):
            raise ValueError("uniforms must be [groups][2 nparams][nshots]")
    grad = np.zeros(max(1, P))
    N.check(N.lib().qs_faithful_gradient(circuit.handle, N.dptr(p), obs.handle, code, int(nshots),
                                         N.dptr(u) if u is not None else None, ctypes.c_void_p(states.data_ptr()),
                                         ctypes.c_void_p(work.data_ptr()) if work is not None else None,
                                         _stream_ptr(), N.dptr(grad)))
    return grad[:P]


def mmd_gradient(circuit: Circuit, params, target, sigma: float, dtype=torch.complex128, nshots: int = 0,
                 uniforms=None, device="cuda"):
    """(loss, grad) of the MMD loss of the circuit's output distribution against target
    (2^n probabilities), Gaussian kernel of bandwidth sigma on basis indices; exact, or
    from nshots samples per register with uniforms [2 nparams + 1][nshots]."""
    P = circuit.nparams
    p = _params_array(params, P)
    code = _dtype_code(dtype)
    q = np.ascontiguousarray(np.asarray(target, dtype=np.float64))
    if q.size != (1 << circuit.nqubits):
        raise ValueError("target must have 2^n entries")
    states = torch.empty((2 * P + 1) << circuit.nqubits, dtype=_TORCH_DTYPE[code], device=device)
    u = None
    if nshots > 0:
        u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
        if u.shape != (2 * P + 1, nshots):
            raise ValueError("uniforms must be [2 nparams + 1][nshots]")
    grad = np.zeros(max(1, P))
    loss = np.zeros(1)
    N.check(N.lib().qs_mmd_gradient(circuit.handle, N.dptr(p), N.dptr(q), float(sigma), code, int(nshots),
                                    N.dptr(u) if u is not None else None, ctypes.c_void_p(states.data_ptr()),
                                    _stream_ptr(), N.dptr(grad), N.dptr(loss)))
    return float(loss[0]), grad[:P]


def observable_csr(obs: Observable, nqubits: int, device="cuda"):
    """mat(O) as CSR on the device: (rowptr int64 [2^n + 1], cols int64 [nnz], vals complex128 [nnz])."""
    L = N.lib()
    dim = 1 << nqubits
    rowptr = torch.empty(dim + 1, dtype=torch.int64, device=device)
    scratch = torch.empty(dim // 1024 + 2, dtype=torch.int64, device=device)
    nnz = ctypes.c_int64(0)
    N.check(L.qs_observable_csr_rows(obs.handle, int(nqubits), ctypes.c_void_p(rowptr.data_ptr()),
                                     ctypes.c_void_p(scratch.data_ptr()), ctypes.byref(nnz), _stream_ptr()))
    cols = torch.empty(max(1, nnz.value), dtype=torch.int64, device=device)
    vals = torch.empty(max(1, nnz.value), dtype=torch.complex128, device=device)
    N.check(L.qs_observable_csr_fill(obs.handle, int(nqubits), ctypes.c_void_p(rowptr.data_ptr()),
                                     ctypes.c_void_p(cols.data_ptr()), ctypes.c_void_p(vals.data_ptr()), _stream_ptr()))
    return rowptr, cols[:nnz.value], vals[:nnz.value]


def batch_autotune(circuits, observables, state: State, params: torch.Tensor, grad: bool = True, reps: int = 2):
    """Tile size (qubits) at which the batched program runs fastest on this state, and
    {tile: ms}.  The state's amplitudes are overwritten."""
    L = N.lib()
    nreg = len(circuits)
    ch = (ctypes.c_void_p * nreg)(*[c.handle.value for c in circuits])
    oh = (ctypes.c_void_p * nreg)(*[o.handle.value for o in observables])
    loss = torch.empty(nreg, dtype=torch.float64, device=params.device)
    g = torch.empty_like(params) if grad else None
    best = ctypes.c_int(0)
    cap = 8
    nc = ctypes.c_int(cap)
    tiles = np.zeros(cap, np.int32)
    ms = np.zeros(cap)
    N.check(L.qs_batch_autotune(nreg, ctypes.cast(ch, ctypes.POINTER(ctypes.c_void_p)),
                                ctypes.cast(oh, ctypes.POINTER(ctypes.c_void_p)), state.handle,
                                ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                ctypes.c_void_p(g.data_ptr()) if g is not None else None, int(reps),
                                ctypes.byref(best), ctypes.byref(nc), tiles.ctypes.data_as(N._PI32), N.dptr(ms)))
    return best.value, {int(tiles[i]): float(ms[i]) for i in range(min(nc.value, cap))}


def batch_autotune_shape(circuits, observables, state: State, params: torch.Tensor, grad: bool = True,
                         precise: bool = False, reps: int = 2):
    """Fusion width (phase qubits) and tile size at which the batched program runs fastest
    on this state (qs_batch_autotune_ex): (tile, phase_qubits, {(tile, phase): ms}).  The
    state's amplitudes are overwritten."""
    L = N.lib()
    nreg = len(circuits)
    ch = (ctypes.c_void_p * nreg)(*[c.handle.value for c in circuits])
    oh = (ctypes.c_void_p * nreg)(*[o.handle.value for o in observables])
    loss = torch.empty(nreg, dtype=torch.float64, device=params.device)
    g = torch.empty_like(params) if grad else None
    bt, bp = ctypes.c_int(0), ctypes.c_int(0)
    cap = 16
    nc = ctypes.c_int(cap)
    tiles = np.zeros(cap, np.int32)
    phases = np.zeros(cap, np.int32)
    ms = np.zeros(cap)
    N.check(L.qs_batch_autotune_ex(nreg, ctypes.cast(ch, ctypes.POINTER(ctypes.c_void_p)),
                                   ctypes.cast(oh, ctypes.POINTER(ctypes.c_void_p)),
                                   N.QS_BATCH_PRECISE if precise else 0, state.handle,
                                   ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                   ctypes.c_void_p(g.data_ptr()) if g is not None else None, int(reps),
                                   ctypes.byref(bt), ctypes.byref(bp), ctypes.byref(nc), tiles.ctypes.data_as(N._PI32),
                                   phases.ctypes.data_as(N._PI32), N.dptr(ms)))
    return bt.value, bp.value, {(int(tiles[i]), int(phases[i])): float(ms[i]) for i in range(min(nc.value, cap))}
