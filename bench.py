#!/usr/bin/env python3
"""Benchmark of the GB300 state-vector hot path.

Headline: single-gate HBM throughput at n = 25 qubits (2^25 amplitudes,
complex64, Haar-random state from seed 0).  Suite: X, H, T, Rx(0.7) on every
qubit, CNOT on (0,1), (11,12), (23,24), Toffoli on (0,1->2), (22,23->24); each
gate applied 100 times.  One step = 100 rounds of the 105-gate suite (10,500
single-gate launches; a gate's repetitions are interleaved with the rest of the
suite so a small touched set never stays in L2).  value = algorithmic bytes /
device time, where a gate's algorithmic bytes are read + write of every 32-byte
sector holding at least one amplitude the gate changes.

Extra keys: the same sweep in complex128, the roofline of the dominant kernel
(live CUDA events per launch), clocks sampled during the timed region, e2e
through host buffers, and the FP64 oracle timed on the host cores.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

N_QUBITS = 25
REPS = 100
SEED = 0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ byte model

def touched_mask(g) -> int:
    """Bits whose value is fixed for every amplitude the gate changes."""
    m = 0
    for c in g.ctrl_locs:
        m |= 1 << c
    if g.name in ("T", "TDG", "S", "SDG", "Z", "SHIFT"):  # diagonal with one non-unit entry
        m |= 1 << g.locs[0]
    return m


def gate_bytes(g, n: int, amp_bytes: int) -> int:
    """Read + write of every 32-byte sector holding at least one changed amplitude."""
    per_sector = 32 // amp_bytes
    low = per_sector.bit_length() - 1   # bits inside a sector
    hi_fixed = bin(touched_mask(g) >> low).count("1")
    sectors = 1 << (n - low - hi_fixed)
    return 2 * 32 * sectors


def kernel_class(g) -> str:
    if g.name in ("X",):
        return "swap1"
    if g.name in ("T", "TDG", "S", "SDG", "Z", "SHIFT", "RZ"):
        return "diag1"
    return "dense1"


# ------------------------------------------------------------------ clocks

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ GPU sweep

class Sweep:
    """Pre-marshalled single-gate launches through the C ABI (qs_apply_named)."""

    def __init__(self, st, suite):
        from paper_1912_10877_gb300 import _native as N
        self.N = N
        self.L = N.lib()
        self.h = st.handle
        self.calls = []
        for label, g in suite:
            self.calls.append((N.GATE_KIND[g.name], len(g.locs), N.i32(g.locs), N.i32([]),
                               len(g.ctrl_locs), N.i32(g.ctrl_locs), N.i32(g.ctrl_vals),
                               float(g.theta or 0.0)))

    def round(self, events=None, base=0):
        f = self.L.qs_apply_named
        h = self.h
        for i, c in enumerate(self.calls):
            rc = f(h, *c)
            if rc:
                self.N.check(rc)
            if events is not None:
                events[base + i].record()


def run_sweep(dtype_name: str, steps: int, warmup: int, dev, with_events: bool):
    import torch
    from paper_1912_10877_gb300 import qsim
    tdt = torch.complex64 if dtype_name == "c64" else torch.complex128
    amp = 8 if dtype_name == "c64" else 16
    n = N_QUBITS
    suite = W.single_gate_suite(n)
    psi = W.haar_state(n, SEED)
    st = qsim.State(n, dtype=tdt)
    st.upload(psi)
    sw = Sweep(st, suite)
    bytes_round = sum(gate_bytes(g, n, amp) for _, g in suite)
    for _ in range(warmup):
        for _ in range(REPS):
            sw.round()
    torch.cuda.synchronize()
    nl = len(suite)
    events = None
    if with_events:
        events = [torch.cuda.Event(enable_timing=True) for _ in range(REPS * nl + 1)]
    per_class_t = {}
    per_class_b = {}
    t_total = 0.0
    for s in range(steps):
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record()
        if events is not None:
            events[0].record()
        for r in range(REPS):
            sw.round(events, 1 + r * nl)
        end.record()
        torch.cuda.synchronize()
        t_total += start.elapsed_time(end) / 1e3
        if events is not None:
            for r in range(REPS):
                for i, (_, g) in enumerate(suite):
                    k = 1 + r * nl + i
                    dt = events[k - 1].elapsed_time(events[k]) / 1e3
                    c = kernel_class(g)
                    per_class_t[c] = per_class_t.get(c, 0.0) + dt
                    per_class_b[c] = per_class_b.get(c, 0) + gate_bytes(g, n, amp)
    total_bytes = bytes_round * REPS * steps
    res = {"seconds": t_total, "bytes": total_bytes, "gbs": total_bytes / t_total / 1e9,
           "launches": nl * REPS * steps, "per_class": {}}
    for c in per_class_t:
        res["per_class"][c] = {"seconds": per_class_t[c], "gbs": per_class_b[c] / per_class_t[c] / 1e9,
                               "launches": None}
    res["state"] = st
    res["psi"] = psi
    res["sweep"] = sw
    res["bytes_round"] = bytes_round
    return res


def run_sizes_leg(ns=(26, 28, 30, 32), rounds: int = 2, hbm_peak: float = 0.0):
    """The complex64 single-gate suite at larger registers (one launch per gate and
    round, per-launch CUDA events).  The state starts as |+...+> made on the device
    (H on every qubit of |0...0>): a host-made Haar state of 2^32 amplitudes would
    need 64 GiB of host memory, and the kernels' time does not depend on the values."""
    import torch
    from paper_1912_10877_gb300 import qsim
    out = {}
    for n in ns:
        suite = W.single_gate_suite(n)
        st = qsim.State(n, dtype=torch.complex64)
        st.reset()
        for q in range(n):
            st.apply(W.Gate("H", (q,)))
        sw = Sweep(st, suite)
        sw.round()                                   # warm-up round
        nl = len(suite)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(rounds * nl + 1)]
        torch.cuda.synchronize()
        ev[0].record()
        for r in range(rounds):
            sw.round(ev, 1 + r * nl)
        torch.cuda.synchronize()
        t, b, worst = {}, {}, None
        for r in range(rounds):
            for i, (_, g) in enumerate(suite):
                dt = ev[r * nl + i].elapsed_time(ev[r * nl + i + 1]) / 1e3
                c = kernel_class(g)
                gb = gate_bytes(g, n, 8)
                t[c] = t.get(c, 0.0) + dt
                b[c] = b.get(c, 0) + gb
                if r == rounds - 1:
                    v = gb / dt / 1e9
                    if worst is None or v < worst[0]:
                        worst = (v, f"{g.name} {g.locs}" + (f" ctrl {g.ctrl_locs}" if g.ctrl_locs else ""))
        total_t, total_b = sum(t.values()), sum(b.values())
        out[str(n)] = {"gbs": round(total_b / total_t / 1e9, 1),
                       "frac": round(total_b / total_t / 1e9 / hbm_peak, 4) if hbm_peak else None,
                       "per_class_gbs": {c: round(b[c] / t[c] / 1e9, 1) for c in t},
                       "slowest_gate": {"gbs": round(worst[0], 1), "gate": worst[1]},
                       "state_gib": (1 << n) * 8 / 2 ** 30, "launches": rounds * nl}
        del sw, st
        torch.cuda.empty_cache()
    return {"metric": "single-gate suite HBM GB/s at larger registers (complex64)", "unit": "GB/s",
            "rounds": rounds, "init": "|+...+> made on the device", "sizes": out}


def run_e2e(res, steps: int):
    """Same sweep through host buffers: pinned H2D of the input, the sweep, D2H of the result."""
    import torch
    from paper_1912_10877_gb300 import _native as N
    st, sw = res["state"], res["sweep"]
    host_in = torch.from_numpy(res["psi"].astype(np.complex64 if st.dtype_code == N.QS_C64 else np.complex128))
    host_in = host_in.pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    L = N.lib()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        N.check(L.qs_state_upload(st.handle, ctypes.c_void_p(host_in.data_ptr())))
        for _ in range(REPS):
            sw.round()
        N.check(L.qs_state_download(st.handle, ctypes.c_void_p(host_out.data_ptr())))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nb = host_in.numel() * host_in.element_size()
    return {"value": res["bytes_round"] * REPS * steps / dt / 1e9, "unit": "GB/s",
            "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb}


def traffic_for(kernel: str):
    """(per-launch DRAM bytes, note) from a committed ncu summary: the bytes only if the
    kernel's source file is unchanged since the capture, else None and a note naming the
    stale figure."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        entry = t[kernel]
        src = open(os.path.join(ROOT, "paper_1912_10877_gb300", "csrc", entry["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest() != entry["sha256"]:
            return None, (f"{entry['source']} changed since the capture of {entry['dram_bytes_per_launch']} bytes "
                          f"per launch ({entry.get('changed_since', 'see profiles/traffic.json')})")
        return entry["dram_bytes_per_launch"], None
    except Exception:
        return None, "no committed capture"


# ------------------------------------------------------------------ batched registers (fwd + grad)

BATCH_NREG, BATCH_LO, BATCH_HI, BATCH_DEPTH = 1024, 10, 18, 20


def batch_workload():
    counts = W.batch_qubit_counts(BATCH_NREG, BATCH_LO, BATCH_HI, seed=0)
    specs = W.batch_variational(counts, BATCH_DEPTH, seed=0)
    return counts, specs


def run_batch_leg(steps: int, warmup: int, compare: bool = True, world: int = 1, rank: int = 0):
    """1024 registers, n ~ U{10..18}, Rz Rx Rz + CNOT ladder x 20 layers each, <sum Z_i Z_{i+1}>:
    forward + reversible gradient of every register in ONE persistent launch (complex64).
    Two paths, each at the program shape (fusion width = register qubits per phase, tile size)
    the autotuner picks: the FP32 path, and the precise path (compensated complex64 forward,
    double-float uncompute).  With N ranks the registers are split by cost (no data-path
    collective), each rank runs its share, the time is the slowest rank's and the losses are
    gathered.  Comparator (single rank): the unfused gate-by-gate complex128 path (one kernel per
    gate per register, per-gate FP64 adjoint), all 1024 registers on preallocated states,
    device-timed; and the same with each register's forward replayed from a CUDA graph."""
    import torch
    from paper_1912_10877_gb300 import qsim
    from paper_1912_10877_gb300 import dist as D
    counts_all, specs_all = batch_workload()
    mine = D.partition_registers(counts_all, world)[rank]
    counts = [counts_all[r] for r in mine]
    specs = [specs_all[r] for r in mine]
    circs = [qsim.Circuit(g, int(n)) for n, (g, _) in zip(counts, specs)]
    obs = [qsim.Observable(W.zz_chain(int(n))) for n in counts]
    st = qsim.State([int(n) for n in counts], dtype=torch.complex64)
    params = torch.tensor(np.concatenate([p for _, p in specs]), dtype=torch.float64, device="cuda")
    # ALU roofline: the method's minimal FP32 flops per batch.  Forward per layer and qubit:
    # the fused Rz Rx Rz, one complex 2x2 = 2 complex multiply-adds = 16 flops per amplitude.
    # Backward per layer and qubit, rotation by rotation: uncompute psi and lambda (Rz diagonal
    # and Rx real-diagonal / imaginary off-diagonal: 6 flops per amplitude each, x 2 states)
    # plus Im<lambda|G|psi> (4 per amplitude): 3 x 16 = 48.  CNOTs move amplitudes (0 flops);
    # lambda = O psi and <O> are lower order.  Total 64 flops per amplitude, layer and qubit.
    flops = sum(float(BATCH_DEPTH * int(n) * 64) * (1 << int(n)) for n in counts_all)
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12  # TFLOP/s: SMs x FP32 FMA/clk x 2 flops x max SM clock
    loss = torch.empty(len(mine), dtype=torch.float64, device="cuda")
    grad = torch.empty(int(params.numel()), dtype=torch.float64, device="cuda")
    paths = {}
    for name, precise in (("fp32", False), ("precise", True)):
        tile, phase, shapes = qsim.batch_autotune_shape(circs, obs, st, params, grad=True, precise=precise, reps=1)
        prog = qsim.BatchProgram(circs, obs, tile_qubits=tile, phase_qubits=phase, precise=precise)
        for _ in range(warmup):
            prog.run(st, params, grad=True, loss=loss, grad_out=grad)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            prog.run(st, params, grad=True, loss=loss, grad_out=grad)
        e1.record()
        torch.cuda.synchronize()
        t = D.max_over_ranks(e0.elapsed_time(e1) / 1e3 / steps)
        losses = D.gather_per_register(loss.cpu().numpy(), mine, BATCH_NREG)
        assert np.all(np.isfinite(losses)), "a register's loss is missing"
        paths[name] = {"value": round(BATCH_NREG / t, 1), "ms_per_batch": round(1e3 * t, 3),
                       "tile_qubits": tile, "phase_qubits": phase,
                       "autotune_ms": {f"{k[0]}q tile/{k[1]}q phase": round(v, 2) for k, v in shapes.items()}}
        del prog
    t = paths["fp32"]["ms_per_batch"] / 1e3
    res = {"metric": "batched fwd+grad circuits/s", "value": paths["fp32"]["value"], "unit": "circuits/s",
           "roofline": {"bound": "alu", "achieved": round(flops / t / 1e12, 2), "peak": round(fp32_peak, 1),
                        "unit": "TFLOP/s", "frac": round(flops / t / 1e12 / fp32_peak, 4),
                        "peak_kind": "derived: 152 SMs x 128 FP32 FMA/clk x 2 flops x 2.07 GHz",
                        "flops_per_batch": flops},
           "ms_per_batch": paths["fp32"]["ms_per_batch"],
           "dtype": "c64 (f32 gates and uncompute; f64 reductions above warp level)",
           "precise": dict(paths["precise"], dtype="c64 forward with compensated matrices (f32), double-float "
                                                    "uncompute, f64 reductions"),
           "fusion": {k: {"tile_qubits": v["tile_qubits"], "phase_qubits": v["phase_qubits"]} for k, v in paths.items()},
           "autotune_ms": {k: v["autotune_ms"] for k, v in paths.items()},
           "config": {"workload": f"{BATCH_NREG} registers, n ~ U{{{BATCH_LO}..{BATCH_HI}}} seed 0, Rz.Rx.Rz + "
                                  f"CNOT ladder x {BATCH_DEPTH} layers, <sum Z_i Z_i+1> (open)",
                      "total_amplitudes": int(sum(1 << int(n) for n in counts_all)), "launches_per_batch": 2,
                      "ranks": world, "split": "registers by cost 2^n (LPT), losses gathered"}}
    if compare and world == 1:
        res["gate_by_gate_c128"] = run_c128_comparator(counts, specs, circs, obs)
        for k in ("fp32", "precise"):
            res[f"vs_gate_by_gate_c128_{k}"] = round(paths[k]["value"] / res["gate_by_gate_c128"]["value"], 1)
    return res


def run_c128_comparator(counts, specs, circs, obs):
    """The plain complex128 path on the batched workload: per register, one kernel per gate
    (unfused) forward from |0..0> and the per-gate FP64 reversible adjoint, on states
    allocated before the timed region; CUDA events around all 1024 registers (host launch
    overhead included, as it is part of that path).  Variant: each register's forward
    captured once as a CUDA graph and replayed."""
    import torch
    from paper_1912_10877_gb300 import qsim
    states = [qsim.State(int(n), dtype=torch.complex128) for n in counts]
    works = {int(n): qsim.backward_work(int(n)) for n in set(int(n) for n in counts)}
    params = [p for _, p in specs]

    def direct():
        for r in range(len(counts)):
            states[r].reset()
            states[r].apply_circuit(circs[r], params[r], fused=False)
            qsim.backward(states[r], circs[r], params[r], obs[r], work=works[int(counts[r])])

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    direct()
    t_direct = timed(direct)
    graphs = []
    for r in range(len(counts)):
        states[r].reset()
        graphs.append(qsim.CapturedCircuit(states[r], circs[r], params[r], fused=False))

    def captured():
        for r in range(len(counts)):
            states[r].reset()
            graphs[r].replay()
            qsim.backward(states[r], circs[r], params[r], obs[r], work=works[int(counts[r])])

    captured()
    t_graph = timed(captured)
    best = min(t_direct, t_graph)
    return {"value": round(len(counts) / best, 2), "unit": "circuits/s", "seconds": round(best, 3),
            "seconds_direct": round(t_direct, 3), "seconds_forward_graphs": round(t_graph, 3),
            "registers": len(counts), "timing": "CUDA events, states and work buffers preallocated"}


# ------------------------------------------------------------------ differentiation and large registers

def run_diff_leg(steps: int, warmup: int):
    """n = 20, 100 layers of Rz Rx Rz on every qubit + CNOT ring (8000 gates, 6000 angles),
    transverse-field Ising loss.  (a) complex64 forward with checkpoints every 10 layers and
    the FP64 reversible uncompute (qs_backward); (b) the tile engine: fused forward and the
    FP32 tiled backward (qs_backward_tiled)."""
    import torch
    from paper_1912_10877_gb300 import qsim
    n, depth = 20, 100
    gates, params = W.variational(n, depth, "ring", seed=0)
    circ = qsim.Circuit(gates, n)
    obs = qsim.Observable(W.tfim(n))
    every = 10 * 4 * n
    st = qsim.State(n, dtype=torch.complex64)
    ck = qsim.checkpoint_buffer(st, circ, every)
    work = qsim.backward_work(n)

    def fp64_path():
        st.reset()
        qsim.apply_circuit_ckpt(st, circ, params, every, ck)
        return qsim.backward(st, circ, params, obs, every, ck, work)

    def tiled_path():
        st.reset()
        st.apply_circuit(circ, params, tiles=True)
        return qsim.backward_tiled(st, circ, params, obs)

    out = {}
    for name, fn in (("fp64_uncompute_ckpt10", fp64_path), ("tiled_fp32", tiled_path)):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        torch.cuda.synchronize()
        out[name] = round((time.perf_counter() - t0) / steps, 4)
    # the backward alone (its FP64 uncompute is the bound): forward once, then time qs_backward
    st.reset()
    qsim.apply_circuit_ckpt(st, circ, params, every, ck)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    qsim.backward(st, circ, params, obs, every, ck, work)
    tb = time.perf_counter() - t0
    # FP64 roofline of the backward: per rotation and amplitude pair, uncompute psi and lambda
    # (Rz^dag: two complex-by-phase products, 6 flops each, per state; Rx^dag: c a + i s b, 6 flops
    # per amplitude, per state) and Im<lambda|G|psi> (8 flops per pair): 32 FP64 flops per pair,
    # 16 per amplitude; CNOTs move amplitudes (0 flops)
    fp64_flops = 6000 * 16.0 * (1 << n)
    fp64_peak = 1.25  # TFLOP/s, nominal FP64 of GB300
    return {"metric": "fwd+grad seconds (n=20, 8000 gates, 6000 angles)", "unit": "s",
            "value": out["fp64_uncompute_ckpt10"], "tiled_fp32_value": out["tiled_fp32"],
            "backward_s": round(tb, 4),
            "roofline": {"bound": "alu", "kernel": "FP64 reversible uncompute (k_adjoint_param1 / k_adjoint_param)",
                         "achieved": round(fp64_flops / tb / 1e12, 3), "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": round(fp64_flops / tb / 1e12 / fp64_peak, 4), "flops": fp64_flops,
                         "peak_kind": "nominal FP64 rate of GB300 (1.25 TFLOP/s)"},
            "forward": "complex64, 1-qubit gates with compensated matrices rounded once (checkpointed path)",
            "passes": qsim.schedule_info(circ)[0], "higher_is_better": False,
            "config": {"workload": "n=20, 100 x (Rz Rx Rz per qubit + CNOT ring), <sum ZZ + sum X>, seed 0",
                       "checkpoints": f"every {every} gates (10 layers)"}}


def run_large_leg(steps: int, warmup: int):
    """n = 32 (32 GiB complex64): QFT with swap network on a seeded basis state, depth-20
    brickwork of Rz + Haar SU(2) + CZ, reversible gradient of <Z_1> w.r.t. the 640 angles.
    The QFT runs on the tile engine (6 passes: its controlled phases fuse); the brickwork
    forward runs both ways, on the tile engine and as fused 5-qubit blocks (dense ones on
    the tensor cores), and the faster one counts; the gradient runs on the tile engine."""
    import torch
    from paper_1912_10877_gb300 import qsim
    n, depth = 32, 20
    x = W.random_basis(n, seed=0)
    qc = qsim.Circuit(W.qft(n, swaps=True), n)
    bgates, bparams = W.brickwork(n, depth, seed=0)
    bc = qsim.Circuit(bgates, n, nparams=len(bparams))
    obs = qsim.Observable(W.z_on(0))
    st = qsim.State(n, dtype=torch.complex64)
    b = ctypes.c_size_t()
    from paper_1912_10877_gb300 import _native as Nn
    Nn.check(Nn.lib().qs_backward_tiled_work_bytes(n, ctypes.byref(b)))
    work = torch.empty(b.value, dtype=torch.uint8, device="cuda")
    qp, bp = qsim.schedule_info(qc)[0], qsim.schedule_info(bc)[0]
    nblocks = len(qsim.circuit_blocks(bc, bparams, 5, matrices=False))

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    def run_once():
        st.reset([x])
        tq = timed(lambda: st.apply_circuit(qc, tiles=True))
        tb_tiles = timed(lambda: st.apply_circuit(bc, bparams, tiles=True))
        st.reset([x])
        timed(lambda: st.apply_circuit(qc, tiles=True))
        tb_blocks = timed(lambda: st.apply_circuit(bc, bparams, blocks=5))
        tg = timed(lambda: qsim.backward_tiled(st, bc, bparams, obs, work=work))
        # the same gradient over 5-qubit blocks, from the same forward state
        st.reset([x])
        timed(lambda: st.apply_circuit(qc, tiles=True))
        timed(lambda: st.apply_circuit(bc, bparams, blocks=5))
        tgb = timed(lambda: qsim.backward_blocks(st, bc, bparams, obs, kmax=5, work=work))
        return tq, tb_tiles, tb_blocks, tg, tgb

    for _ in range(warmup):
        run_once()
    acc = np.zeros(5)
    for _ in range(steps):
        acc += np.array(run_once())
    tq, tbt, tbb, tgt, tgb = acc / steps
    tf = tq + min(tbt, tbb)
    tg = min(tgt, tgb)
    S = 8 << n
    return {"metric": "n=32 QFT + depth-20 brickwork forward and <Z_1> gradient", "unit": "s",
            "value": round(tf + tg, 4), "forward_s": round(tf, 4), "backward_s": round(tg, 4),
            "qft_tiles": {"seconds": round(tq, 4), "passes": qp, "gbs": round(qp * 2 * S / tq / 1e9, 1)},
            "brickwork_tiles": {"seconds": round(tbt, 4), "passes": bp, "gbs": round(bp * 2 * S / tbt / 1e9, 1)},
            "brickwork_blocks5": {"seconds": round(tbb, 4), "passes": nblocks,
                                  "gbs": round(nblocks * 2 * S / tbb / 1e9, 1)},
            "brickwork_forward_used": "blocks5" if tbb < tbt else "tiles",
            "gradient_tiles": {"seconds": round(tgt, 4), "passes": bp, "gbs": round(bp * 4 * S / tgt / 1e9, 1)},
            "gradient_blocks5": {"seconds": round(tgb, 4), "blocks": nblocks,
                                 "gbs": round(nblocks * 6 * S / tgb / 1e9, 1)},
            "gradient_used": "blocks5" if tgb < tgt else "tiles",
            "gates": {"qft": len(W.qft(n, swaps=True)), "brickwork": len(bgates)},
            "roofline": {"bound": "hbm", "kernel": "whole workload (QFT passes, 5-qubit block passes, block gradient)",
                         "achieved": round(large_bytes(qp, nblocks, S, tbb < tbt, bp, tgb < tgt) / (tf + tg) / 1e9, 1),
                         "peak": hbm_peak_of(), "unit": "GB/s",
                         "frac": round(large_bytes(qp, nblocks, S, tbb < tbt, bp, tgb < tgt) / (tf + tg) / 1e9
                                       / hbm_peak_of(), 4),
                         "bytes": large_bytes(qp, nblocks, S, tbb < tbt, bp, tgb < tgt),
                         "model": "QFT passes x 2S + forward block (or tile) passes x 2S + gradient blocks x 6S "
                                  "(Gram reads psi and lambda, the adjoint reads and writes both; tile-pass "
                                  "gradient: 4S per pass); S = 32 GiB"},
            "higher_is_better": False,
            "config": {"workload": "n=32 c64, QFT+swaps on basis state (seed 0), brickwork depth 20 (seed 0), "
                                   "grad of <Z_1> wrt 640 angles", "state_gib": 32}}


def hbm_peak_of() -> float:
    return peaks()[0]


def large_bytes(qft_passes: int, nblocks: int, S: int, blocks_forward: bool, tile_passes: int,
                blocks_gradient: bool = True) -> float:
    """Algorithmic HBM bytes of the large workload as run: every pass over the 32 GiB state
    reads and writes it once (2S); a block of the gradient reads psi and lambda for its Gram
    and reads and writes both in its adjoint (6S); a tile pass of the gradient reads and
    writes psi and lambda (4S)."""
    fwd = (nblocks if blocks_forward else tile_passes) * 2 * S
    grad = nblocks * 6 * S if blocks_gradient else tile_passes * 4 * S
    return float(qft_passes * 2 * S + fwd + grad)


def run_small_leg(reps: int = 50):
    """The small workload (n = 12, complex128, |0..0>, 10 layers of Rz Rx Rz + CNOT ladder,
    <sum Z_i Z_{i+1}> open): launch-bound.  Per circuit: the gate-by-gate path (one
    launch per gate), the default path (single-qubit runs fused on the host), and the
    default path's launches captured once as a CUDA graph and replayed."""
    import torch
    from paper_1912_10877_gb300 import qsim
    n = 12
    gates, params = W.variational(n, 10, "ladder", seed=0)
    circ = qsim.Circuit(gates, n)
    obs = qsim.Observable(W.zz_chain(n))
    st = qsim.State(n, dtype=torch.complex128)

    def per_circuit(fn):
        for _ in range(3):
            st.reset()
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) * 1e3 / reps

    t_unf = per_circuit(lambda: st.apply_circuit(circ, params, fused=False))
    t_def = per_circuit(lambda: st.apply_circuit(circ, params))
    st.reset()
    cap = qsim.CapturedCircuit(st, circ, params)
    t_graph = per_circuit(cap.replay)
    blocks = {}
    for k in (3, 4, 5):
        st.reset()
        capk = qsim.CapturedCircuit(st, circ, params, blocks=k)
        blocks[str(k)] = {"graph_replay_us": round(per_circuit(capk.replay), 1),
                          "launches": len(qsim.circuit_blocks(circ, params, k, matrices=False))}
    st.reset()
    cap.replay()
    e = float(st.expect(obs)[0])
    # the whole circuit and <sum ZZ> in one cooperative launch, per block width and grid size
    one = {}
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for k in (3, 4, 5):
        for grid in (0, 64, 32):
            t = per_circuit(lambda: qsim.run_one_launch(st, circ, params, kmax=k, obs=obs, grid_ctas=grid, out=out))
            one[f"k{k}_grid{grid or 'sms'}"] = round(t, 1)
    st.reset()
    qsim.run_one_launch(st, circ, params, kmax=4, obs=obs, out=out)
    e1 = float(out.item())
    best_one = min(one.values())
    best = min([t_def, t_graph, best_one] + [b["graph_replay_us"] for b in blocks.values()])
    return {"metric": "small variational circuit latency (n=12, complex128)", "unit": "us per circuit",
            "value": round(best, 1), "gate_by_gate_us": round(t_unf, 1), "default_us": round(t_def, 1),
            "graph_replay_us": round(t_graph, 1), "blocks_graph_replay": blocks,
            "one_launch_us": {"best": best_one, "by_shape": one,
                              "note": "circuit and <sum ZZ> in one cooperative launch (fused blocks of k qubits, "
                                      "grid barrier between blocks)"},
            "roofline": {"bound": "latency", "achieved": round(best, 1), "unit": "us per circuit",
                         "note": "a 64 KiB register: launch and barrier latency and the FP64 rate of the SMs it "
                                 "reaches bound it, not HBM"},
            "gates": len(gates), "expectation": e, "expectation_one_launch": e1, "higher_is_better": False}


def run_sharded_leg(n: int = 24, nglobal: int = 2, depth: int = 4):
    """The qubit-sharded register on one GPU (all 2^g shards in this process, exchanges as
    device copies): the variational circuit forward, <sum ZZ + sum X> and the reversible
    gradient (complex128 working copies, one library adjoint step per gate and shard),
    against the same work on one unsharded complex64 register (per-gate FP64 adjoint)."""
    import torch
    from paper_1912_10877_gb300 import qsim
    from paper_1912_10877_gb300.sharded import ShardedState
    gates, params = W.variational(n, depth, "ring", seed=0)
    terms = W.tfim(n)
    circ = qsim.Circuit(gates, n)

    def sharded():
        sh = ShardedState(n, nglobal, torch.complex64)
        sh.apply_circuit(circ, params)
        loss, grad = sh.backward(circ, params, terms)
        torch.cuda.synchronize()
        return sh.exchanges

    def plain():
        st = qsim.State(n, dtype=torch.complex64)
        st.reset()
        st.apply_circuit(circ, params, fused=False)
        qsim.backward(st, circ, params, qsim.Observable(terms))
        torch.cuda.synchronize()

    sharded()
    plain()
    t0 = time.perf_counter()
    ex = sharded()
    ts = time.perf_counter() - t0
    t0 = time.perf_counter()
    plain()
    tp = time.perf_counter() - t0
    return {"metric": f"qubit-sharded register fwd+grad seconds (n={n}, {1 << nglobal} shards, one GPU)", "unit": "s",
            "value": round(ts, 4), "unsharded_s": round(tp, 4), "exchanges": ex, "gates": len(gates),
            "params": len(params), "higher_is_better": False,
            "note": "host wall clock; shards exchange halves by device copies in one process"}


def run_faithful_leg(n: int = 10, depth: int = 4, nshots: int = 1024):
    """Shot-based faithful gradients (Eq. shiftrule) of the transverse-field Ising energy for
    the n = 10 variational circuit: 2P shifted circuits run as one batch (complex64, the
    batched engine), each sampled nshots times per measurement-basis group; and the MMD
    loss gradient of the same circuit's Born distribution against a seeded target."""
    import torch
    from paper_1912_10877_gb300 import qsim
    gates, params = W.variational(n, depth, "ladder", seed=0)
    circ = qsim.Circuit(gates, n)
    obs = qsim.Observable(W.tfim(n))
    P = len(params)
    G = qsim.observable_groups(obs)
    u = W.rng(5).random((G, 2 * P, nshots))
    um = W.rng(6).random((2 * P + 1, nshots))
    target = W.rng(7).random(1 << n)
    target /= target.sum()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    t_shot = timed(lambda: qsim.faithful_gradient(circ, params, obs, dtype=torch.complex64, nshots=nshots, uniforms=u))
    t_exact = timed(lambda: qsim.faithful_gradient(circ, params, obs, dtype=torch.complex64))
    t_mmd = timed(lambda: qsim.mmd_gradient(circ, params, target, 2.0, dtype=torch.complex64, nshots=nshots,
                                            uniforms=um))
    return {"metric": f"faithful (parameter-shift) gradient seconds, n={n}, {P} parameters", "unit": "s",
            "value": round(t_shot, 4), "exact_expectation_s": round(t_exact, 4), "mmd_shots_s": round(t_mmd, 4),
            "shots_per_circuit": nshots, "groups": G, "shifted_circuits": 2 * P, "higher_is_better": False,
            "note": "host wall clock around one call (launches, sampling and the host reduction included)"}


def run_matrix_leg(n: int = 20, reps: int = 5):
    """mat(heisenberg(n)) (periodic) as a CSR matrix on the device: row pointers (count +
    scan) and the fill, timed together; the paper reports 6.33 s for n = 20 on a laptop."""
    import torch
    from paper_1912_10877_gb300 import qsim
    obs = qsim.Observable(W.heisenberg(n))
    qsim.observable_csr(obs, n)
    torch.cuda.synchronize()
    ts = []
    nnz = 0
    for _ in range(reps):
        t0 = time.perf_counter()
        rowptr, cols, vals = qsim.observable_csr(obs, n)
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
        nnz = int(cols.numel())
        del rowptr, cols, vals
    t = float(np.median(ts))
    return {"metric": f"mat(heisenberg({n})) CSR construction", "unit": "s", "value": round(t, 5), "nnz": nnz,
            "bytes_written": nnz * 24 + ((1 << n) + 1) * 8, "higher_is_better": False,
            "paper_context": "6.330 s for mat(heisenberg(20)) on a laptop (Sec. Matrix Representation and AD Performance)"}


def run_tiles_leg(n: int = 26, reps: int = 3):
    """Tile engine at n = 26 (complex64, 512 MiB): QFT + swaps on a basis state and a
    depth-20 brickwork, forward passes and the brickwork's reversible gradient of <Z_1>;
    per-pass HBM GB/s (each pass reads and writes the state once; the gradient moves
    psi and lambda).  Also the brickwork as 5-qubit blocks.  For profiling captures."""
    import torch
    from paper_1912_10877_gb300 import qsim
    x = W.random_basis(n, seed=0)
    qc = qsim.Circuit(W.qft(n, swaps=True), n)
    bgates, bparams = W.brickwork(n, 20, seed=0)
    bc = qsim.Circuit(bgates, n, nparams=len(bparams))
    obs = qsim.Observable(W.z_on(0))
    st = qsim.State(n, dtype=torch.complex64)
    b = ctypes.c_size_t()
    from paper_1912_10877_gb300 import _native as Nn
    Nn.check(Nn.lib().qs_backward_tiled_work_bytes(n, ctypes.byref(b)))
    work = torch.empty(b.value, dtype=torch.uint8, device="cuda")
    qp, bp = qsim.schedule_info(qc)[0], qsim.schedule_info(bc)[0]
    nblocks = len(qsim.circuit_blocks(bc, bparams, 5, matrices=False))
    S = 8 << n

    def timed(fn):
        ts = []
        for _ in range(reps):
            st.reset([x])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return float(np.median(ts))

    tq = timed(lambda: st.apply_circuit(qc, tiles=True))
    tb = timed(lambda: st.apply_circuit(bc, bparams, tiles=True))
    tk = timed(lambda: st.apply_circuit(bc, bparams, blocks=5))
    tg = timed(lambda: qsim.backward_tiled(st, bc, bparams, obs, work=work))
    wb = torch.empty(S, dtype=torch.uint8, device="cuda")
    tgb = timed(lambda: qsim.backward_blocks(st, bc, bparams, obs, kmax=5, work=wb))
    return {"metric": f"tile engine per-pass HBM GB/s at n={n}", "unit": "GB/s",
            "qft": {"passes": qp, "seconds": round(tq, 5), "gbs": round(qp * 2 * S / tq / 1e9, 1)},
            "brickwork": {"passes": bp, "seconds": round(tb, 5), "gbs": round(bp * 2 * S / tb / 1e9, 1)},
            "brickwork_blocks5": {"passes": nblocks, "seconds": round(tk, 5), "gbs": round(nblocks * 2 * S / tk / 1e9, 1)},
            "brickwork_gradient": {"passes": bp, "seconds": round(tg, 5), "gbs": round(bp * 4 * S / tg / 1e9, 1),
                                   "note": "timed on the reset state (the timing, not the values, matters here)"},
            "brickwork_gradient_blocks5": {"blocks": nblocks, "seconds": round(tgb, 5),
                                           "gbs_model": "per block: Gram reads psi, lambda; uncompute r+w both",
                                           "gbs": round(nblocks * 6 * S / tgb / 1e9, 1)}}


def run_tc_leg(reps: int = 20):
    """Dense 4- and 5-qubit blocks at n = 25 (complex64, Haar state): the tensor-core
    kernel (3xTF32 tcgen05 GEMM) against the CUDA-core kernel, per target placement.
    Bytes per launch: the state read and written once (2 x 2^25 x 8 B); L2 flushed
    between launches.  The tensor-core flop rate counts the 3 TF32 products."""
    import torch
    from paper_1912_10877_gb300 import qsim
    n = N_QUBITS
    rs = np.random.default_rng(SEED)
    st = qsim.State(n, dtype=torch.complex64)
    st.upload(W.haar_state(n, SEED))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    byts = 2 * (1 << n) * 8
    out = {}
    for k in (4, 5):
        d = 1 << k
        a = rs.standard_normal((d, d)) + 1j * rs.standard_normal((d, d))
        q, r = np.linalg.qr(a)
        U = q * (np.diag(r) / np.abs(np.diag(r)))
        for place, locs in (("low", tuple(range(k))), ("high", tuple(range(n - k, n))),
                            ("mixed", (1, 7, 13, 19, 24)[:k])):
            g = W.Gate("MATRIX", locs, matrix=U)
            row = {}
            for mode, name in ((2, "tensor"), (0, "cuda_core")):
                qsim.set_tensor_cores(mode)
                for _ in range(3):
                    st.apply(g)
                torch.cuda.synchronize()
                ts = []
                for _ in range(reps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    st.apply(g)
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1) / 1e3)
                t = float(np.median(ts))
                row[name + "_gbs"] = round(byts / t / 1e9, 1)
                if mode == 2:
                    w = 2 * d
                    tiles = (1 << (n - k)) / 128
                    row["tensor_tf32_tflops"] = round(tiles * 3 * 2 * 128 * w * w / t / 1e12, 1)
            st.sync()
            out[f"k{k}_{place}"] = row
    qsim.set_tensor_cores(1)
    return {"metric": "dense k-qubit block HBM GB/s at n=25, tensor cores vs CUDA cores", "unit": "GB/s",
            "placements": {"low": "targets 0..k-1", "high": "targets n-k..n-1", "mixed": "targets (1,7,13,19,24)[:k]"},
            "results": out, "launches": 2 * 2 * 3 * (reps + 3)}


# ------------------------------------------------------------------ CPU baseline (oracle)

METRIC = "gate HBM GB/s at n=25 (single-gate suite, complex64)"


def suite_config(world: int) -> dict:
    return {"workload": "single-gate suite: X,H,T,Rx(0.7) on each of 25 qubits, 3 CNOT, 2 Toffoli; "
                        "100 reps each; Haar state n=25 seed 0",
            "n": N_QUBITS, "reps": REPS, "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (256 MiB state); reps interleaved across the suite"}


def oracle_baseline(budget_s: float = 15.0):
    """The FP64 oracle, as it stands, applying suite gates to the n = 25 state on the host cores.
    Sample: gates of the suite in order, one application each, until ~budget_s of CPU work."""
    import oracle
    n = N_QUBITS
    suite = W.single_gate_suite(n)
    psi = W.haar_state(n, SEED)
    order = list(range(0, len(suite), 7)) + [i for i in range(len(suite)) if i % 7]
    t0 = time.perf_counter()
    nbytes = 0
    done = 0
    for i in order:
        _, g = suite[i]
        psi = oracle.apply_circuit(psi, n, [g])
        nbytes += gate_bytes(g, n, 8)   # the metric's byte model: the same gate on a complex64 state
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": nbytes / dt / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": f"{done} single-gate applications of the n=25 suite, {dt:.1f} s on {cores} OpenMP threads; "
                      f"the oracle computes in FP64, bytes are counted as for the complex64 state of the metric"}, dt


def oracle_configs_baseline(budget_s: float = 10.0):
    """The FP64 oracle, as it stands, on the host cores for the other workloads (bounded
    samples, each stated): the small circuit in full; the batch on a 32-register subset
    scaled to 1024 (extrapolated); the differentiation workload's forward + adjoint
    gradient over its first layers, scaled to the 100 layers (extrapolated)."""
    import oracle
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {}
    # small: n = 12, complex128, 10 layers, <sum ZZ>
    gates, params = W.variational(12, 10, "ladder", seed=0)
    t0 = time.perf_counter()
    reps = 0
    while reps < 1 or time.perf_counter() - t0 < 1.0:
        oracle.expect(oracle.apply_circuit(oracle.zero_state(12), 12, gates, params), 12, W.zz_chain(12))
        reps += 1
    dt = (time.perf_counter() - t0) / reps
    out["small"] = {"value": round(dt * 1e6, 1), "unit": "us per circuit", "cores": cores, "kind": "oracle",
                    "sample": f"the full n=12 circuit and <sum ZZ>, {reps} runs"}
    # batch: registers spread over the size range, forward + gradient each
    counts, specs = batch_workload()
    order = np.argsort(counts, kind="stable")
    spread = [int(order[i]) for i in np.linspace(0, len(order) - 1, 32).astype(int)]
    pick = [spread[(i // 2) if i % 2 == 0 else (31 - i // 2)] for i in range(32)]  # small and large alternate
    t0 = time.perf_counter()
    done = 0
    for r in pick:
        n = int(counts[r])
        g, p = specs[r]
        oracle.gradient(oracle.zero_state(n), n, g, p, W.zz_chain(n))
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    # scale by cost 2^n of the registers done against the whole batch
    cost_done = sum(2.0 ** int(counts[r]) for r in pick[:done])
    cost_all = float(sum(2.0 ** int(n) for n in counts))
    t_all = dt * cost_all / cost_done
    out["batched"] = {"value": round(BATCH_NREG / t_all, 3), "unit": "circuits/s", "cores": cores, "kind": "oracle",
                      "sample": f"forward + adjoint gradient of {done} registers spread over n=10..18 in {dt:.1f} s, "
                                f"scaled by their share of the batch's cost sum 2^n (extrapolated)"}
    # differentiation: n = 20, first layers of the 100-layer circuit, scaled
    n, layers = 20, 2
    gates, params = W.variational(n, layers, "ring", seed=0)
    t0 = time.perf_counter()
    oracle.gradient(oracle.zero_state(n), n, gates, params, W.tfim(n))
    dt = time.perf_counter() - t0
    out["differentiation"] = {"value": round(dt * 100 / layers, 2), "unit": "s", "cores": cores, "kind": "oracle",
                              "sample": f"forward + adjoint gradient of the first {layers} of 100 layers at n=20 in "
                                        f"{dt:.1f} s, scaled x{100 // layers} (extrapolated)"}
    return out


def summary_of(line: dict) -> dict:
    """The headline figures of every leg in one short object (printed last in the line)."""
    def g(d, *ks):
        for k in ks:
            d = d.get(k) if isinstance(d, dict) else None
        return d

    out = {"headline_gbs": line.get("value"), "headline_frac": g(line, "roofline", "frac"),
           "headline_traffic": g(line, "roofline", "traffic"), "e2e_gbs": g(line, "e2e", "value")}
    b = line.get("batched")
    if isinstance(b, dict):
        out["batched_circuits_s"] = b.get("value")
        out["batched_frac"] = g(b, "roofline", "frac")
        out["batched_shape"] = g(b, "fusion", "fp32")
        out["batched_precise_circuits_s"] = g(b, "precise", "value")
        out["batched_precise_shape"] = g(b, "fusion", "precise")
        out["gate_by_gate_c128_circuits_s"] = g(b, "gate_by_gate_c128", "value")
        out["batched_vs_c128"] = b.get("vs_gate_by_gate_c128_fp32")
        out["batched_precise_vs_c128"] = b.get("vs_gate_by_gate_c128_precise")
    d = line.get("differentiation")
    if isinstance(d, dict):
        out["differentiation_s"] = d.get("value")
        out["differentiation_fp64_frac"] = g(d, "roofline", "frac")
    L = line.get("large")
    if isinstance(L, dict):
        out["large_s"] = L.get("value")
        out["large_hbm_frac"] = g(L, "roofline", "frac")
    sm = line.get("small")
    if isinstance(sm, dict):
        out["small_us"] = sm.get("value")
    for k in ("sharded", "faithful", "matrix"):
        v = line.get(k)
        if isinstance(v, dict):
            out[f"{k}_s"] = v.get("value")
    cb = line.get("cpu_baseline_configs")
    if isinstance(cb, dict):
        out["oracle"] = {k: v.get("value") for k, v in cb.items()}
    return out


# ------------------------------------------------------------------ main

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def main():
    global REPS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-c128", action="store_true")
    ap.add_argument("--no-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-tc", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-matrix", action="store_true")
    ap.add_argument("--no-sizes", action="store_true")
    ap.add_argument("--leg", default="all",
                    choices=["all", "tc", "batch", "diff", "large", "tiles", "small", "matrix", "sizes", "sharded",
                             "faithful"],
                    help="run one secondary leg alone and print its JSON (profiling captures)")
    ap.add_argument("--tc-reps", type=int, default=20, help="timed launches per tensor-core configuration")
    ap.add_argument("--reps", type=int, default=REPS, help="repetitions per gate (profiling runs use 1)")
    args = ap.parse_args()
    REPS = args.reps
    world, rank, local = dist_setup(args)
    hbm_peak, peak_kind = peaks()

    if args.impl == "reference":
        if rank != 0:
            return 0
        import oracle
        oracle.build()
        vals = []
        for _ in range(args.warmup):
            oracle_baseline(budget_s=2.0)
        t_all = 0.0
        last = None
        for _ in range(args.steps):
            last, dt = oracle_baseline(budget_s=10.0)
            vals.append(last["value"])
            t_all += dt
        v = float(np.mean(vals))
        line = {"impl": "reference", "metric": METRIC, "value": v,
                "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_all / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": suite_config(1),
                "cpu_baseline": {"value": v, "unit": "GB/s", "cores": last["cores"], "kind": "oracle",
                                 "sample": last["sample"]},
                "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1912_10877_gb300 import lib
    lib()

    if args.leg != "all":
        legs = {"tc": lambda: run_tc_leg(args.tc_reps),
                "batch": lambda: run_batch_leg(max(1, args.steps), max(1, args.warmup), compare=not args.no_compare,
                                               world=world, rank=rank),
                "diff": lambda: run_diff_leg(1, 1), "large": lambda: run_large_leg(1, 1),
                "tiles": lambda: run_tiles_leg(), "small": lambda: run_small_leg(),
                "matrix": lambda: run_matrix_leg(), "sizes": lambda: run_sizes_leg(hbm_peak=hbm_peak),
                "sharded": lambda: run_sharded_leg(), "faithful": lambda: run_faithful_leg()}
        out = legs[args.leg]()
        if rank == 0:
            print(json.dumps(out))
        return 0

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # --- headline: complex64 sweep with live per-launch events
    barrier()
    clocks = Clocks(local)
    clocks.start()
    c64 = run_sweep("c64", args.steps, args.warmup, local, with_events=True)
    clk = clocks.stop()
    barrier()
    from paper_1912_10877_gb300 import dist as D
    t = D.max_over_ranks(c64["seconds"])
    value = c64["bytes"] * world / t / 1e9
    e2e = None if args.no_e2e else run_e2e(c64, max(1, args.steps))
    if world > 1 and e2e:
        e2e["value"] *= world
    # dominant kernel: largest share of device time
    pc = c64["per_class"]
    dom = max(pc, key=lambda c: pc[c]["seconds"])
    kname = {"dense1": "k_gate1<float, 5|6, *> (OP_REAL1: H; OP_RXLIKE1: Rx)", "swap1": "k_gate1<float, 2, *> (OP_SWAP1: X, CNOT, Toffoli)",
             "diag1": "k_diag1<float> (T: touched half only)"}[dom]
    achieved = pc[dom]["gbs"]
    roof = {"kernel": kname, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak,
            "peak_kind": f"{peak_kind} (copy GB/s)", "unit": "GB/s", "frac": round(achieved / hbm_peak, 4),
            "traffic": None,
            "per_class_gbs": {c: round(v["gbs"], 1) for c, v in pc.items()},
            "per_class_share": {c: round(v["seconds"] / sum(x["seconds"] for x in pc.values()), 4)
                                for c, v in pc.items()}}
    roof["traffic"], note = traffic_for(dom + "_c64")
    if note:
        roof["traffic_note"] = note
    del c64
    extra = {}
    # secondary single-GPU legs run at N = 1 only (scaling runs time the headline and the sharded batch)
    solo = world == 1
    if not args.no_c128 and solo:
        c128 = run_sweep("c128", max(1, args.steps // 3), max(1, args.warmup // 3), local, with_events=True)
        extra["c128_sweep"] = {"value": round(c128["gbs"], 1), "unit": "GB/s", "steps": max(1, args.steps // 3),
                               "per_class_gbs": {c: round(v["gbs"], 1) for c, v in c128["per_class"].items()},
                               "note": "complex128 FP64 arithmetic; dense 2x2 is FP64-ALU bound on GB300"}
        del c128
    if not args.no_batch:
        extra["batched"] = run_batch_leg(max(1, args.steps), max(1, args.warmup), compare=not args.no_compare,
                                         world=world, rank=rank)
    if not args.no_tc and solo:
        extra["tensor_core_blocks"] = run_tc_leg(args.tc_reps)
    if solo and not args.no_small:
        extra["small"] = run_small_leg()
    if solo and not args.no_matrix:
        extra["matrix"] = run_matrix_leg()
        extra["sharded"] = run_sharded_leg()
        extra["faithful"] = run_faithful_leg()
    if solo and not args.no_sizes:
        extra["single_gate_sizes"] = run_sizes_leg(hbm_peak=hbm_peak)
    if not args.no_large and solo:
        extra["differentiation"] = run_diff_leg(1, 1)
        extra["large"] = run_large_leg(1, 1)
    launches = REPS * len(W.single_gate_suite(N_QUBITS)) * args.steps
    line = {"metric": METRIC, "value": round(value, 1),
            "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * t / args.steps, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64 (f32)", "data": "synthetic",
            "config": suite_config(world),
            "roofline": roof, "clocks": clk, "e2e": e2e, "gpu_launches": launches}
    line.update(extra)
    if rank == 0 and not args.no_baseline and world == 1:
        cb, _ = oracle_baseline(budget_s=15.0)
        line["cpu_baseline"] = cb
        line["cpu_baseline_configs"] = oracle_configs_baseline()
    line["summary"] = summary_of(line)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
