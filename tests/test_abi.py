"""CPU checks of the C ABI: the library loads, exports every entry point the
header declares, its struct layouts match the binding, and host-only argument
validation reports errors (no GPU needed, no kernel is launched)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "qsim.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_1912_10877_gb300 import build as B
    B.build()
    from paper_1912_10877_gb300 import _native as N
    return N.lib()


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 20
    from paper_1912_10877_gb300 import _native as N
    for name in names:
        assert hasattr(L, name), f"{name} not exported"
        assert name in N.SIGNATURES, f"{name} has no binding signature"


def test_struct_layout_matches_binding(tmp_path):
    from paper_1912_10877_gb300 import _native as N
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "qsim.h"\n'
        "int main(void){\n"
        ' printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(qs_gate_desc), offsetof(qs_gate_desc, param),'
        " offsetof(qs_gate_desc, ctrl_mask), offsetof(qs_gate_desc, mat_offset), offsetof(qs_gate_desc, theta),"
        " sizeof(qs_pauli_term));\n return 0; }\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    G = N.GateDesc
    want = [ctypes.sizeof(G), G.param.offset, G.ctrl_mask.offset, G.mat_offset.offset, G.theta.offset,
            ctypes.sizeof(N.PauliTerm)]
    assert got == want


def _circuit(L, gates, n, nparams=0):
    from paper_1912_10877_gb300 import _native as N
    arr = (N.GateDesc * max(1, len(gates)))(*gates)
    h = ctypes.c_void_p()
    rc = L.qs_circuit_create(n, arr, len(gates), None, 0, nparams, ctypes.byref(h))
    return rc, h


def test_host_validation_errors(L):
    from paper_1912_10877_gb300 import _native as N
    g = N.GateDesc()
    g.kind, g.nlocs, g.param = N.GATE_KIND["X"], 1, -1
    g.locs[0] = 3
    rc, h = _circuit(L, [g], 3)  # loc 3 on a 3-qubit circuit
    assert rc == N.QS_EINVAL and b"out of range" in L.qs_last_error()
    g.locs[0] = 1
    g.ctrl_mask = 1 << 1  # control equals target
    rc, h = _circuit(L, [g], 3)
    assert rc == N.QS_EINVAL and b"control" in L.qs_last_error()
    g.ctrl_mask = 0
    g.kind, g.param = N.GATE_KIND["H"], 0  # H takes no parameter
    rc, h = _circuit(L, [g], 3, nparams=1)
    assert rc == N.QS_EINVAL
    g.kind = N.GATE_KIND["RX"]
    rc, h = _circuit(L, [g], 3, nparams=1)
    assert rc == N.QS_OK
    cnt = ctypes.c_int()
    assert L.qs_checkpoint_count(h, 1, ctypes.byref(cnt)) == 0 and cnt.value == 0
    assert L.qs_circuit_destroy(h) == 0
    b = ctypes.c_size_t()
    assert L.qs_backward_work_bytes(20, ctypes.byref(b)) == 0 and b.value == 2 * 16 * (1 << 20)
    nq = (ctypes.c_int32 * 3)(10, 12, 11)
    assert L.qs_state_bytes(3, nq, N.QS_C64, ctypes.byref(b)) == 0 and b.value == 8 * (1024 + 4096 + 2048)
    assert L.qs_state_bytes(1, (ctypes.c_int32 * 1)(0), N.QS_C64, ctypes.byref(b)) == N.QS_EINVAL
    assert L.qs_state_bytes(1, nq, 7, ctypes.byref(b)) == N.QS_EINVAL


def test_observable_handle_roundtrip(L):
    from paper_1912_10877_gb300 import _native as N
    terms = (N.PauliTerm * 2)()
    terms[0].coeff, terms[0].z_mask = 1.0, 0b11
    terms[1].coeff, terms[1].x_mask = 0.5, 0b1
    h = ctypes.c_void_p()
    assert L.qs_observable_create(terms, 2, ctypes.byref(h)) == 0
    assert L.qs_observable_destroy(h) == 0
    assert L.qs_observable_create(None, 2, ctypes.byref(h)) == N.QS_EINVAL


def test_package_has_no_cpu_fallback():
    # the product package never imports the oracle
    pkg = os.path.join(ROOT, "paper_1912_10877_gb300")
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            src = open(os.path.join(pkg, fn)).read()
            assert "import oracle" not in src and "from oracle" not in src, fn


def test_host_gate_matrices_match_the_oracle(L):
    """qs_circuit_gate_matrices (host code of the library) against the oracle's own
    gate definitions, and the generator against a finite difference of U:
    dU/dtheta = -i c H U for U = exp(-i theta c H)."""
    import oracle
    import workloads as W
    from paper_1912_10877_gb300 import qsim
    oracle.build()
    gates = [W.Gate("H", (0,)), W.Gate("T", (1,)), W.Gate("RX", (2,), param=0), W.Gate("RY", (0,), (1,), (0,), param=1),
             W.Gate("RZ", (1,), param=2), W.Gate("SHIFT", (0,), (2,), (1,), param=3), W.Gate("PHASE", (1,), param=4),
             W.Gate("ROT", (0, 2), paulis="XZ", param=5), W.Gate("SWAP", (1, 2)), W.Gate("SDG", (2,))]
    params = np.array([0.3, -1.2, 2.5, 0.7, 1.9, -0.4])
    c = qsim.Circuit(gates, 3)
    h = 1e-6
    for i, g in enumerate(gates):
        theta = params[g.param] if g.param is not None else 0.0
        U = c.gate_matrices(i, params)
        assert np.max(np.abs(U - oracle.gate_matrix(g, theta))) < 1e-15, g.name
        if g.param is None:
            with pytest.raises(Exception):
                c.gate_matrices(i, params, generator=True)
            continue
        _, G, cf = c.gate_matrices(i, params, generator=True)
        dU = (oracle.gate_matrix(g, theta + h) - oracle.gate_matrix(g, theta - h)) / (2 * h)
        assert np.max(np.abs(dU - (-1j * cf * G @ U))) < 1e-9, g.name


def test_host_validation_of_gate_records(L):
    # malformed gate records are refused at circuit creation (QS_EINVAL), before any device work
    from paper_1912_10877_gb300 import _native as N

    def gate(kind, locs, ctrl=0, vals=0, param=-1, paulis=(), mat_offset=0):
        g = N.GateDesc()
        g.kind, g.nlocs, g.param = N.GATE_KIND[kind], len(locs), param
        for j, q in enumerate(locs):
            g.locs[j] = q
        for j, p in enumerate(paulis):
            g.paulis[j] = p
        g.ctrl_mask, g.ctrl_vals, g.mat_offset = ctrl, vals, mat_offset
        return g

    wide = gate("MATRIX", [0, 1, 2, 3, 4])
    wide.nlocs = 6
    bad = [
        ([wide], 8, 0),                                         # more targets than QS_MAXK
        ([gate("X", [])], 8, 0),                                # no target
        ([gate("SWAP", [2, 2])], 8, 0),                         # repeated target
        ([gate("SWAP", [2])], 8, 0),                            # SWAP needs two targets
        ([gate("X", [0], ctrl=1 << 8)], 8, 0),                  # control outside the register
        ([gate("RX", [0], param=3)], 8, 2),                     # parameter index past nparams
        ([gate("ROT", [0, 1], paulis=(1, 4))], 8, 0),           # not a Pauli code
        ([gate("MATRIX", [0], mat_offset=0)], 8, 0),            # matrix pool too small (empty)
    ]
    for gates, n, nparams in bad:
        rc, h = _circuit(L, gates, n, nparams=nparams)
        assert rc == N.QS_EINVAL, (gates[0].kind, L.qs_last_error())
    for n in (0, N.QS_MAXQ + 1 if hasattr(N, "QS_MAXQ") else 41):
        rc, h = _circuit(L, [], n)
        assert rc == N.QS_EINVAL
    # host-only planners: argument ranges
    rc, h = _circuit(L, [gate("H", [0]), gate("X", [3], ctrl=1)], 8)
    assert rc == N.QS_OK
    cnt = ctypes.c_int()
    assert L.qs_circuit_tile_order(h, 8, ctypes.byref(cnt), None, None) == N.QS_EINVAL
    assert L.qs_circuit_tile_order(h, 9, ctypes.byref(cnt), None, None) == N.QS_OK and cnt.value == 2
    assert L.qs_circuit_destroy(h) == 0
    rc, h = _circuit(L, [gate("H", [0])], 4)
    assert L.qs_circuit_tile_order(h, 0, ctypes.byref(cnt), None, None) == N.QS_EUNSUPPORTED
    assert L.qs_circuit_destroy(h) == 0
