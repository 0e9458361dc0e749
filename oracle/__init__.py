"""FP64 CPU oracle for the state-vector hot path (Yao.jl, arXiv 1912.10877).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the bench's
``cpu_baseline`` / ``--impl reference`` legs are the only callers.  Nothing in
the product package imports this module; the CUDA path fails loudly without its
own extension instead of falling back to this code.

The arithmetic lives in ``qsim_oracle.c`` (plain C, complex double), compiled
by ``build()`` into ``liboracle.so`` next to this file.  This wrapper only
marshals the shared gate-list format of ``workloads`` into the C structs and
composes oracle calls (parameter-shift and finite-difference gradients are
compositions of expectation calls).

Functions and the passages they follow:
  apply_circuit   Sec. "Representing Quantum Circuits" (apply!, chain order) and
                  Sec. "Performance" (general multi-control instruction)
  apply_dagger    Sec. "Manipulating Quantum Circuits" (dagger rules)
  expect          Sec. "Forward Mode" (expect of sums of Pauli strings)
  gradient        Sec. "Reverse Mode", Eqs. apply-back / outer-product
  adjoint_step    one gate of that walk
  shift_gradient  Eq. shiftrule (only for uncontrolled Pauli rotations)
  fd_gradient     central finite differences of ``expect``
  sample/collapse Sec. "Instructions on Quantum Registers" (measure / measure!),
                  with the deterministic sampling contract stated in the C file
  sample_seeded   the same with uniforms from SplitMix64 (Steele, Lea and Flood
                  2014), the library's seeded-measurement contract
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsim_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MAXK, MAXC, MAXOPS = 5, 16, 64
_KIND = {"I": 0, "X": 1, "Y": 2, "Z": 3, "H": 4, "S": 5, "SDG": 6, "T": 7, "TDG": 8,
         "RX": 9, "RY": 10, "RZ": 11, "SHIFT": 12, "PHASE": 13, "SWAP": 14, "ROT": 15,
         "MATRIX": 16}
_PAULI = {"X": 1, "Y": 2, "Z": 3}


class _Gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("k", ctypes.c_int32),
                ("locs", ctypes.c_int32 * MAXK), ("nctrl", ctypes.c_int32),
                ("ctrl_locs", ctypes.c_int32 * MAXC), ("ctrl_vals", ctypes.c_int32 * MAXC),
                ("param", ctypes.c_int32), ("paulis", ctypes.c_int32 * MAXK),
                ("mat_offset", ctypes.c_int64), ("theta", ctypes.c_double)]


class _Term(ctypes.Structure):
    _fields_ = [("coeff", ctypes.c_double), ("nops", ctypes.c_int32),
                ("locs", ctypes.c_int32 * MAXOPS), ("paulis", ctypes.c_int32 * MAXOPS)]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, OpenMP over basis indices).

    QSIM_ORACLE_LIB names a prebuilt copy to load instead (the mutation tests
    load copies with planted mistakes this way, each in its own process)."""
    alt = os.environ.get("QSIM_ORACLE_LIB")
    if alt:
        return alt
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fcx-limited-range", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_apply_circuit.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(_Gate),
                                        ctypes.c_int, dp, ctypes.c_void_p, ctypes.c_int]
        L.orc_expect.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(_Term),
                                 ctypes.c_int, dp]
        L.orc_apply_observable.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                           ctypes.POINTER(_Term), ctypes.c_int]
        L.orc_gradient.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(_Gate),
                                   ctypes.c_int, dp, ctypes.c_int, ctypes.c_void_p,
                                   ctypes.POINTER(_Term), ctypes.c_int, dp, dp]
        L.orc_sample.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_int64)]
        L.orc_collapse.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64]
        L.orc_gate_matrix.argtypes = [ctypes.POINTER(_Gate), ctypes.c_double, ctypes.c_void_p,
                                      ctypes.c_void_p]
        L.orc_pairwise_sum.argtypes = [dp, ctypes.c_int64]
        L.orc_pairwise_sum.restype = ctypes.c_double
        for f in ("orc_apply_circuit", "orc_expect", "orc_apply_observable", "orc_gradient",
                  "orc_sample", "orc_gate_matrix"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _marshal_gates(gates):
    arr = (_Gate * max(1, len(gates)))()
    mats = []
    off = 0
    for i, g in enumerate(gates):
        s = arr[i]
        s.kind = _KIND[g.name]
        s.k = len(g.locs)
        if s.k < 1 or s.k > MAXK or len(g.ctrl_locs) > MAXC:
            raise ValueError("gate arity out of range")
        for j, l in enumerate(g.locs):
            s.locs[j] = l
        s.nctrl = len(g.ctrl_locs)
        for j, (l, v) in enumerate(zip(g.ctrl_locs, g.ctrl_vals)):
            s.ctrl_locs[j] = l
            s.ctrl_vals[j] = v
        s.param = -1 if g.param is None else int(g.param)
        s.theta = 0.0 if g.theta is None else float(g.theta)
        if g.name == "ROT":
            if g.paulis is None or len(g.paulis) != s.k:
                raise ValueError("ROT needs one Pauli per target")
            for j, p in enumerate(g.paulis):
                s.paulis[j] = _PAULI[p]
        if g.name == "MATRIX":
            m = np.ascontiguousarray(g.matrix, dtype=np.complex128)
            if m.shape != (1 << s.k, 1 << s.k):
                raise ValueError("matrix shape does not match the number of targets")
            s.mat_offset = off
            mats.append(m.ravel())
            off += m.size
    pool = np.concatenate(mats) if mats else np.zeros(1, np.complex128)
    return arr, pool


def _marshal_terms(terms):
    arr = (_Term * max(1, len(terms)))()
    for i, (c, ops) in enumerate(terms):
        arr[i].coeff = float(c)
        arr[i].nops = len(ops)
        for j, (l, p) in enumerate(ops):
            arr[i].locs[j] = int(l)
            arr[i].paulis[j] = _PAULI[p]
    return arr


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def _params(params):
    return np.ascontiguousarray(np.zeros(1) if params is None or len(params) == 0 else params,
                                dtype=np.float64)


def zero_state(n: int) -> np.ndarray:
    v = np.zeros(1 << n, np.complex128)
    v[0] = 1.0
    return v


def basis_state(n: int, x: int) -> np.ndarray:
    v = np.zeros(1 << n, np.complex128)
    v[x] = 1.0
    return v


def apply_circuit(psi, n, gates, params=None, dagger=False) -> np.ndarray:
    """Returns a new FP64 state: the gate list applied in order (or its dagger)."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    assert out.shape == (1 << n,)
    arr, pool = _marshal_gates(gates)
    p = _params(params)
    _check(lib().orc_apply_circuit(out.ctypes.data, n, arr, len(gates), _dp(p), pool.ctypes.data,
                                   1 if dagger else 0), "apply_circuit")
    return out


def apply_dagger(psi, n, gates, params=None) -> np.ndarray:
    return apply_circuit(psi, n, gates, params, dagger=True)


def gate_matrix(g: W.Gate, theta: float = 0.0) -> np.ndarray:
    arr, pool = _marshal_gates([g])
    K = 1 << len(g.locs)
    U = np.zeros((K, K), np.complex128)
    _check(lib().orc_gate_matrix(arr, float(theta), pool.ctypes.data, U.ctypes.data), "gate_matrix")
    return U


def expect(psi, n, terms) -> float:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.zeros(1)
    arr = _marshal_terms(terms)
    _check(lib().orc_expect(psi.ctypes.data, n, arr, len(terms), _dp(out)), "expect")
    return float(out[0])


def apply_observable(psi, n, terms) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    lam = np.zeros_like(psi)
    arr = _marshal_terms(terms)
    _check(lib().orc_apply_observable(lam.ctypes.data, psi.ctypes.data, n, arr, len(terms)),
           "apply_observable")
    return lam


def gradient(psi0, n, gates, params, terms):
    """(loss, dloss/dparams) by the reversible adjoint method of Sec. "Reverse Mode"."""
    psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
    p = _params(params)
    nparams = 0 if params is None else len(params)
    grad = np.zeros(max(1, nparams))
    loss = np.zeros(1)
    arr, pool = _marshal_gates(gates)
    tarr = _marshal_terms(terms)
    _check(lib().orc_gradient(psi0.ctypes.data, n, arr, len(gates), _dp(p), nparams, pool.ctypes.data,
                              tarr, len(terms), _dp(grad), _dp(loss)), "gradient")
    return float(loss[0]), grad[:nparams]


def adjoint_step(psi, lam, n, gate, params, grad):
    """One gate of the reversible adjoint walk (Sec. "Reverse Mode", Eq. apply-back),
    in place on the complex128 arrays psi and lam: grad[gate.param] += 2 c
    Im<lam|H psi> for a parameterised gate, then psi, lam <- U^dag psi, U^dag lam."""
    assert psi.dtype == np.complex128 and lam.dtype == np.complex128 and psi.flags.c_contiguous
    arr, pool = _marshal_gates([gate])
    p = _params(params)
    nparams = 0 if params is None else len(params)
    g = np.ascontiguousarray(grad, dtype=np.float64)
    phi = np.zeros_like(psi)
    im = np.zeros(len(psi))
    _check(lib().orc_adjoint_step(psi.ctypes.data, lam.ctypes.data, phi.ctypes.data, _dp(im), n, arr, _dp(p),
                                  nparams, pool.ctypes.data, _dp(g)), "adjoint_step")
    grad[:] = g


def loss(psi0, n, gates, params, terms) -> float:
    return expect(apply_circuit(psi0, n, gates, params), n, terms)


def shift_gradient(psi0, n, gates, params, terms):
    """Eq. shiftrule: d<O>/dtheta = (<O>(theta+pi/2) - <O>(theta-pi/2)) / 2.  Valid only
    when every use of the parameter is an uncontrolled Pauli rotation (reflexive generator)."""
    for g in gates:
        if g.param is not None and (g.name not in ("RX", "RY", "RZ", "ROT") or g.ctrl_locs):
            raise ValueError("parameter shift needs uncontrolled Pauli rotations")
    params = np.asarray(params, dtype=np.float64)
    out = np.zeros(len(params))
    for i in range(len(params)):
        pp, pm = params.copy(), params.copy()
        pp[i] += math.pi / 2
        pm[i] -= math.pi / 2
        out[i] = 0.5 * (loss(psi0, n, gates, pp, terms) - loss(psi0, n, gates, pm, terms))
    return out


def fd_gradient(psi0, n, gates, params, terms, h=1e-5, which=None):
    """Central finite differences (FP64) of the loss, for the parameters in ``which``."""
    params = np.asarray(params, dtype=np.float64)
    idx = range(len(params)) if which is None else which
    out = {}
    for i in idx:
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        out[i] = (loss(psi0, n, gates, pp, terms) - loss(psi0, n, gates, pm, terms)) / (2 * h)
    return out if which is not None else np.array([out[i] for i in range(len(params))])


def sample(psi, n, u) -> np.ndarray:
    """Basis indices sampled from |psi|^2 with the given uniforms (see the C contract)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    u = np.ascontiguousarray(np.ravel(u), dtype=np.float64)
    out = np.zeros(len(u), np.int64)
    _check(lib().orc_sample(psi.ctypes.data, n, _dp(u), len(u),
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))), "sample")
    return out


def splitmix64(seed: int, k: int) -> int:
    """The k-th output (k >= 1) of SplitMix64 started from ``seed``."""
    f = lib().orc_splitmix64
    f.restype = ctypes.c_uint64
    f.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    return int(f(seed, k))


def seeded_uniforms(seed: int, nreg: int, nshots: int) -> np.ndarray:
    """Uniforms [nreg][nshots] of the seeded measurement: register r's shot j is
    draw k = r * nshots + j + 1 of SplitMix64(seed), u = (x >> 11) * 2^-53."""
    u = np.zeros(nreg * nshots)
    f = lib().orc_seeded_uniforms
    f.restype = None
    f.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
    f(seed, 0, nreg * nshots, _dp(u))
    return u.reshape(nreg, nshots)


def sample_seeded(psi, n, seed: int, nshots: int, reg: int = 0) -> np.ndarray:
    """``sample`` with register ``reg``'s uniforms of the seeded measurement."""
    u = np.zeros(nshots)
    f = lib().orc_seeded_uniforms
    f.restype = None
    f.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
    f(seed, reg * nshots, nshots, _dp(u))
    return sample(psi, n, u)


def collapse(psi, n, x) -> np.ndarray:
    out = np.array(psi, dtype=np.complex128, copy=True)
    lib().orc_collapse(out.ctypes.data, n, int(x))
    return out


def pairwise_sum(v) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return float(lib().orc_pairwise_sum(_dp(v), len(v)))
