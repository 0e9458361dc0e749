"""The bench's algorithmic byte model (read + write of every 32-byte sector that
holds a changed amplitude) against the per-gate table worked out by hand for
the n = 25 single-gate suite (qubits 1-based there, 0-based here), in both
precisions; and the reference arm's line names the GPU line's metric."""
import importlib.util
import os

import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def expected_multiple(g, amp):
    """Bytes of one application in units of the state size S, by hand: the
    gate touches every sector (2S) unless a fixed bit lies above the sector."""
    in_sector = 2 if amp == 8 else 1   # c64: 4 amplitudes (bits 0, 1) per sector; c128: 2 (bit 0)
    fixed = list(g.ctrl_locs)
    if g.name == "T":
        fixed.append(g.locs[0])
    outside = sum(1 for b in fixed if b >= in_sector)
    return 2.0 / (1 << outside)


@pytest.mark.parametrize("amp", [8, 16])
def test_gate_bytes_match_the_hand_table(bench, amp):
    n = 25
    S = (1 << n) * amp
    suite = W.single_gate_suite(n)
    assert len(suite) == 4 * n + 3 + 2
    for label, g in suite:
        assert bench.gate_bytes(g, n, amp) == expected_multiple(g, amp) * S, label
    # the hand table's named cases
    cases = {W.Gate("H", (7,)): 2.0, W.Gate("T", (0,)): 2.0, W.Gate("T", (2,)): 1.0,
             W.cnot(0, 1): 2.0, W.cnot(11, 12): 1.0, W.toffoli(22, 23, 24): 0.5}
    cases[W.Gate("T", (1,))] = 2.0 if amp == 8 else 1.0
    cases[W.toffoli(0, 1, 2)] = 2.0 if amp == 8 else 1.0
    for g, mult in cases.items():
        assert bench.gate_bytes(g, n, amp) == mult * S, (g.name, g.locs, g.ctrl_locs)


def test_reference_arm_uses_the_gpu_metric(bench):
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert src.count('"metric": METRIC') == 2
    assert src.count('"config": suite_config(') == 2
