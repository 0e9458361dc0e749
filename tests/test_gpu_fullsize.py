"""Full-size parity of the single-gate microbenchmark (n = 25, Haar state seed 0),
through qs_apply_named exactly as bench.py launches it.

- one application of every gate type at sampled locations vs the FP64 oracle,
  element by element over the whole 2^25 state;
- 100 applications of every suite gate vs the closed forms the oracle pins fix:
  X, H, CNOT, Toffoli -> identity; T^100 = Z; Rx(0.7)^100 = Rx(70).
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 25
TOL = {"c64": 2e-5, "c128": 1e-12}
TDT = {"c64": torch.complex64, "c128": torch.complex128}


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1912_10877_gb300 import qsim
    return qsim, W.haar_state(N, seed=0)


def apply_reps(qs, st, g, reps):
    from paper_1912_10877_gb300 import _native as Nat
    L = Nat.lib()
    args = (Nat.GATE_KIND[g.name], len(g.locs), Nat.i32(g.locs), Nat.i32([]), len(g.ctrl_locs),
            Nat.i32(g.ctrl_locs), Nat.i32(g.ctrl_vals), float(g.theta or 0.0))
    for _ in range(reps):
        Nat.check(L.qs_apply_named(st.handle, *args))


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_single_application_vs_oracle(env, dt):
    qs, psi = env
    st = qs.State(N, dtype=TDT[dt])
    inp = psi.astype(np.complex64).astype(np.complex128) if dt == "c64" else psi
    sampled = [(l, g) for l, g in W.single_gate_suite(N)
               if g.ctrl_locs or g.locs[0] in (0, 1, 2, 13, 24)]
    for label, g in sampled:
        st.upload(psi)
        apply_reps(qs, st, g, 1)
        got = st.numpy()
        want = oracle.apply_circuit(inp, N, [g])
        assert np.max(np.abs(got - want)) < TOL[dt], label


@pytest.mark.parametrize("dt", ["c64", "c128"])
def test_hundred_repetitions_closed_forms(env, dt):
    qs, psi = env
    st = qs.State(N, dtype=TDT[dt])
    inp = psi.astype(np.complex64).astype(np.complex128) if dt == "c64" else psi
    for label, g in W.single_gate_suite(N):
        st.upload(psi)
        apply_reps(qs, st, g, 100)
        got = st.numpy()
        if g.name in ("X", "H"):
            want = inp
        elif g.name == "T":
            want = oracle.apply_circuit(inp, N, [W.Gate("Z", g.locs)])
        else:
            want = oracle.apply_circuit(inp, N, [W.Gate("RX", g.locs, theta=70.0)])
        assert np.max(np.abs(got - want)) < TOL[dt], label
