"""Seeded synthetic inputs shared by the CUDA path, its tests, the bench and the oracle.

This module describes *what* to simulate: gate lists, parameter vectors, initial
states, observables and the uniform numbers a measurement consumes.  It holds
none of the simulator's arithmetic (no gate matrices are built here, no gate is
applied, nothing is summed), so that the oracle and the CUDA path can both take
their inputs from it without sharing any of the method.

Conventions (paper, Sec. "Instructions on Quantum Registers"): qubits are
little-endian, paper qubit q (1-based) is bit q-1 of the basis index, and a
gate on locs (l_0, ..., l_{k-1}) has matrix index bit j <-> qubit l_j.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# Gate names understood by both sides.  Parameterised names take an angle
# either from the parameter vector (``param``) or fixed (``theta``).
CONST_GATES = ("I", "X", "Y", "Z", "H", "S", "SDG", "T", "TDG", "SWAP")
PARAM_GATES = ("RX", "RY", "RZ", "SHIFT", "PHASE", "ROT")
ALL_GATES = CONST_GATES + PARAM_GATES + ("MATRIX",)


@dataclass(eq=False)
class Gate:
    """One entry of a flat gate list (the paper's put/control blocks, flattened).

    name      : one of ALL_GATES
    locs      : target qubits, 0-based; locs[0] is bit 0 of the gate's own index
    ctrl_locs : control qubits, 0-based
    ctrl_vals : 1 = control on |1>, 0 = inverse control on |0>
    param     : index into the parameter vector, or None
    theta     : fixed angle when ``param`` is None
    paulis    : for ROT, one letter of X/Y/Z per target (generator = tensor product)
    matrix    : for MATRIX, a (2^k, 2^k) complex128 array
    """

    name: str
    locs: tuple
    ctrl_locs: tuple = ()
    ctrl_vals: tuple = ()
    param: int | None = None
    theta: float | None = None
    paulis: str | None = None
    matrix: np.ndarray | None = field(default=None, repr=False)

    def __post_init__(self):
        self.locs = tuple(int(x) for x in self.locs)
        self.ctrl_locs = tuple(int(x) for x in self.ctrl_locs)
        if not self.ctrl_vals:
            self.ctrl_vals = (1,) * len(self.ctrl_locs)
        self.ctrl_vals = tuple(int(x) for x in self.ctrl_vals)
        if self.name not in ALL_GATES:
            raise ValueError(f"unknown gate {self.name}")


def angle(g: Gate, params) -> float:
    """The angle a parameterised gate uses (looked up, not computed)."""
    if g.param is not None:
        return float(params[g.param])
    return 0.0 if g.theta is None else float(g.theta)


# --------------------------------------------------------------------------
# random sources
# --------------------------------------------------------------------------

def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_angles(count: int, seed: int) -> np.ndarray:
    """Angles uniform in [0, 2*pi) from ``seed``."""
    return rng(seed).random(count) * (2.0 * math.pi)


def haar_state(n: int, seed: int) -> np.ndarray:
    """Haar-random normalised state: i.i.d. complex Gaussians, then normalised (complex128)."""
    g = rng(seed)
    dim = 1 << n
    v = g.standard_normal(dim) + 1j * g.standard_normal(dim)
    v /= np.linalg.norm(v)
    return v.astype(np.complex128)


def haar_su2(seed: int) -> np.ndarray:
    """Haar-random SU(2) matrix from a uniformly random unit quaternion."""
    q = rng(seed).standard_normal(4)
    q /= np.linalg.norm(q)
    a = q[0] + 1j * q[1]
    b = q[2] + 1j * q[3]
    return np.array([[a, -np.conj(b)], [b, np.conj(a)]], dtype=np.complex128)


def shot_uniforms(nshots: int, seed: int, nreg: int = 1) -> np.ndarray:
    """The uniform numbers in [0, 1) that ``nshots`` measurements consume, [nreg][nshots]."""
    return rng(seed).random((nreg, nshots))


def random_basis(n: int, seed: int) -> int:
    return int(rng(seed).integers(0, 1 << n))


# --------------------------------------------------------------------------
# circuits
# --------------------------------------------------------------------------

def cnot(c: int, t: int) -> Gate:
    return Gate("X", (t,), (c,), (1,))


def toffoli(c1: int, c2: int, t: int) -> Gate:
    return Gate("X", (t,), (c1, c2), (1, 1))


def variational(n: int, depth: int, entangler: str = "ladder", seed: int = 0,
                params: np.ndarray | None = None):
    """Hardware-efficient ansatz: per layer Rz, Rx, Rz on every qubit, then CNOTs.

    Parameter order: layer -> qubit -> (Rz_1, Rx, Rz_2), applied Rz_1 first.
    ``entangler`` "ladder": CNOT(q, q+1) for q = 0..n-2; "ring" adds CNOT(n-1, 0).
    Returns (gates, params) with params uniform in [0, 2*pi) from ``seed``.
    """
    gates = []
    p = 0
    for _ in range(depth):
        for q in range(n):
            gates.append(Gate("RZ", (q,), param=p))
            gates.append(Gate("RX", (q,), param=p + 1))
            gates.append(Gate("RZ", (q,), param=p + 2))
            p += 3
        for q in range(n - 1):
            gates.append(cnot(q, q + 1))
        if entangler == "ring" and n > 2:
            gates.append(cnot(n - 1, 0))
    if params is None:
        params = uniform_angles(p, seed)
    return gates, np.asarray(params, dtype=np.float64)


def qft(n: int, swaps: bool = False):
    """QFT gate list as the paper's qft listing builds it (Sec. "Representing Quantum
    Circuits"): for each qubit i, H on i, then shift(2*pi/2^(j-i+1)) on i controlled by j
    for every later qubit j.  ``swaps`` appends the swap network SWAP(i, n-1-i)."""
    gates = []
    for i in range(n):
        gates.append(Gate("H", (i,)))
        for j in range(i + 1, n):
            gates.append(Gate("SHIFT", (i,), (j,), (1,), theta=2.0 * math.pi / (2 ** (j - i + 1))))
    if swaps:
        for i in range(n // 2):
            gates.append(Gate("SWAP", (i, n - 1 - i)))
    return gates


def brickwork(n: int, depth: int, seed: int = 0, params: np.ndarray | None = None):
    """Random circuit: per layer, on every qubit Rz(theta) followed by a fixed Haar SU(2)
    matrix V, then CZ on a brickwork pattern (even layers pair (2i, 2i+1), odd layers
    (2i+1, 2i+2)).  One trainable angle per single-qubit gate: n * depth angles."""
    gates = []
    p = 0
    for layer in range(depth):
        for q in range(n):
            gates.append(Gate("RZ", (q,), param=p))
            gates.append(Gate("MATRIX", (q,), matrix=haar_su2(seed * 1_000_003 + p + 1)))
            p += 1
        start = layer % 2
        for q in range(start, n - 1, 2):
            gates.append(Gate("Z", (q + 1,), (q,), (1,)))
    if params is None:
        params = uniform_angles(p, seed)
    return gates, np.asarray(params, dtype=np.float64)


def single_gate_suite(n: int, theta: float = 0.7):
    """Single-gate microbenchmark list: X, H, T, Rx(theta) on every qubit; CNOT on
    (0,1), (n//2-1, n//2), (n-2, n-1); Toffoli on (0,1 -> 2) and (n-3, n-2 -> n-1).
    Returns a list of (label, Gate)."""
    out = []
    for name in ("X", "H", "T"):
        for q in range(n):
            out.append((f"{name}@{q}", Gate(name, (q,))))
    for q in range(n):
        out.append((f"RX@{q}", Gate("RX", (q,), theta=theta)))
    for c in (0, n // 2 - 1, n - 2):
        out.append((f"CNOT@{c},{c + 1}", cnot(c, c + 1)))
    for c in (0, n - 3):
        out.append((f"TOFFOLI@{c},{c + 1},{c + 2}", toffoli(c, c + 1, c + 2)))
    return out


def symad_circuit():
    """The 3-qubit circuit of the paper's App. "Symbolic Differentiation":
    Rx(alpha) on qubit 2, Ry(beta) on qubit 1 controlled by qubit 2, and
    rot(X (x) X, gamma) on qubits (1, 2) (paper numbering; 0-based below)."""
    gates = [
        Gate("RX", (1,), param=0),
        Gate("RY", (0,), (1,), (1,), param=1),
        Gate("ROT", (0, 1), param=2, paulis="XX"),
    ]
    return gates, np.array([0.5, 0.7, 0.8])


def shor_circuit(error_gates):
    """Shor's 9-qubit code (paper App. "Symbolic Computation"): encode, the given error
    gates, decode.  Paper qubit q is loc q-1."""
    c = lambda a, b: cnot(a - 1, b - 1)
    h = lambda a: Gate("H", (a - 1,))
    t2 = lambda a, b, t: toffoli(a - 1, b - 1, t - 1)
    enc = [c(1, 4), c(1, 7), h(1), h(4), h(7), c(1, 2), c(1, 3), c(4, 5), c(4, 6), c(7, 8), c(7, 9)]
    dec = [c(1, 2), c(1, 3), t2(2, 3, 1), c(4, 5), c(4, 6), t2(5, 6, 4), c(7, 8), c(7, 9), t2(8, 9, 7),
           h(1), h(4), h(7), c(1, 4), c(1, 7), t2(4, 7, 1)]
    return enc + list(error_gates) + dec


# --------------------------------------------------------------------------
# observables: lists of (coefficient, ((loc, "X"|"Y"|"Z"), ...))
# --------------------------------------------------------------------------

def zz_chain(n: int, periodic: bool = False):
    terms = [(1.0, ((i, "Z"), (i + 1, "Z"))) for i in range(n - 1)]
    if periodic and n > 2:
        terms.append((1.0, ((n - 1, "Z"), (0, "Z"))))
    return terms


def tfim(n: int, h: float = 1.0):
    """Transverse-field Ising energy: sum of Z_i Z_{i+1} (open) plus h * sum of X_i."""
    return zz_chain(n) + [(h, ((i, "X"),)) for i in range(n)]


def heisenberg(n: int, periodic: bool = True):
    """Sum over bonds of XX + YY + ZZ (periodic bonds reproduce the paper's App. symad)."""
    bonds = [(i, i + 1) for i in range(n - 1)]
    if periodic and n > 2:
        bonds.append((n - 1, 0))
    return [(1.0, ((a, s), (b, s))) for (a, b) in bonds for s in "XYZ"]


def z_on(loc: int):
    return [(1.0, ((loc, "Z"),))]


# --------------------------------------------------------------------------
# batches of uneven registers
# --------------------------------------------------------------------------

def batch_qubit_counts(nreg: int, lo: int, hi: int, seed: int = 0) -> np.ndarray:
    """Register sizes drawn uniformly from {lo, ..., hi}."""
    return rng(seed).integers(lo, hi + 1, size=nreg)


def batch_variational(counts, depth: int, seed: int = 0):
    """Per-register instances of ``variational`` (ladder), register r seeded with seed + r."""
    return [variational(int(n), depth, "ladder", seed=seed + r) for r, n in enumerate(counts)]
