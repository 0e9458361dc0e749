"""Host check of the light-cone reduction the n = 32 large-workload test relies on:
for the brickwork on the QFT of a basis state (a product state), the oracle's loss
and gradient of <Z_1> on the light-cone circuit equal the full circuit's, with
gradient 0 for every angle outside the cone (n = 12, depth 8, oracle only)."""
import math

import numpy as np

import oracle
import workloads as W
from test_gpu_large import light_cone, restricted_gates


def test_light_cone_reduction_is_exact():
    n, depth = 12, 8
    x = W.random_basis(n, seed=3)
    gates, params = W.brickwork(n, depth, seed=3)
    psi0 = oracle.apply_circuit(oracle.basis_state(n, x), n, W.qft(n, swaps=True))
    fl, fg = oracle.gradient(psi0, n, gates, params, W.z_on(0))
    cone = light_cone(gates, n, 0)
    m = len(cone)
    assert cone == set(range(m)) and m == depth
    sub = restricted_gates(gates, cone)
    rx = int(format(x, "0%db" % n)[::-1], 2)
    psi_in = np.array([1.0 + 0j])
    for j in range(m):
        ph = np.exp(2j * np.pi * (rx % (1 << (j + 1))) / (1 << (j + 1)))
        psi_in = np.kron(np.array([1.0, ph]) / math.sqrt(2.0), psi_in)
    sl, sg = oracle.gradient(psi_in, m, sub, params, W.z_on(0))
    used = {g.param for g in sub if g.param is not None}
    outside = np.array([p not in used for p in range(len(params))])
    assert outside.sum() > 0
    assert abs(fl - sl) < 1e-12
    assert np.max(np.abs(fg[outside])) < 1e-12
    assert np.max(np.abs(fg[~outside] - sg[~outside])) < 1e-12
