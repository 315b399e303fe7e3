"""Benchmark: block simulation of a mixed-radix state vector on GB300.

Workload: 18 qubits + 8 qutrits in a seeded wire order (1,719,926,784
amplitudes, 13.76 GB in complex64), 200 gates: 70% Haar-random single-qudit
unitaries, 30% controlled gates (Haar or X_{+1} target, random control wire
and value).  One step = reset to |0...0>, apply the 200 gates (fusion
settings from the autotuner), read the norm.  Metric: amplitude-gate updates
per second (sum over gates of D / prod d_controls).  The 12-qubit + 8-qutrit
Clifford+T-like circuit (500 gates) in complex64 and complex128 and the
other rows of the path (batches, serving, sparse states, ...) are reported
as extra keys of the same line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload on its own GPU (a whole state per GPU has no exchange step); time
is the max over ranks and the value sums the ranks' updates ("weak"
scaling).  ``--impl reference`` times the FP64 CPU oracle on the host cores
on a bounded sample of the same workload (its 20-wire prefix).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = ("18 qubits + 8 qutrits (1,719,926,784 amplitudes), depth 200: 70% Haar single-qudit, "
            "30% controlled (Haar or X_{+1}), seed 2")
BENCH_CIRCUIT = "12 qubits + 8 qutrits (26,873,856 amplitudes), depth 500 hybrid Clifford+T-like mix, seed 1"
METRIC = "amp-gate updates/s"
UNIT = "updates/s"
L2_BYTES = 129e6
PREFIX_WIRES = 20
# FP32 / FP64 vector peaks of GB300 from unit counts and the maximum SM clock:
# 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz; FP64 from NVIDIA's 1.25 TFLOP/s figure.
FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_TFLOPS = 1.25
ALU_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 x 2.07 GHz = 80.5 TFLOP/s (FP64: 1.25 TFLOP/s nominal)"


def bf16_peak() -> float:
    """Dense BF16 tensor peak in TFLOP/s: the measured burst figure (fallback 1900)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f).get("bf16_tflops", 1900.0))
    return 1900.0


def tf32_peak() -> float:
    """Dense TF32 tensor peak in TFLOP/s: the measured bf16 burst figure times the
    nominal TF32/BF16 ratio (1.1 / 2.25)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    bf16 = 1900.0
    if os.path.exists(p):
        with open(p) as f:
            bf16 = float(json.load(f).get("bf16_tflops", bf16))
    return bf16 * 1.1 / 2.25


# ----------------------------------------------------------------------------------------------
# Host logic (tested on CPU)
# ----------------------------------------------------------------------------------------------
def gate_updates(dims, gate) -> int:
    """Logical amplitude updates of one gate: D / prod(d_controls)."""
    D = int(np.prod(np.asarray(dims, dtype=np.int64)))
    for c in gate.controls:
        D //= dims[c]
    return D


def circuit_updates(circ) -> int:
    return sum(gate_updates(circ.dims, g) for g in circ.gates)


def algorithmic_bytes(plan: dict, amp_bytes: int) -> int:
    """Bytes a gate must read and write: every touched row of every visited class, once each way."""
    return 2 * amp_bytes * int(plan["classes"]) * int(plan["touched_rows"])


def method_flops(plan: dict, U) -> float:
    """Floating-point work of one gate as the method states it (a complex
    multiply-add is 8 flops, a complex product 6): a dense P x P gate costs
    8 P flops per amplitude of every visited class; a diagonal (phase) gate 6
    per amplitude it changes; a permutation nothing when every non-zero is 1
    (data movement only), else 6 per amplitude it changes.  ``plan`` is
    ``qd_plan_gate``'s record (kind 0 dense, 1 diagonal, 2 permutation)."""
    U = np.asarray(U)
    P = U.shape[0]
    classes, rows = float(plan["classes"]), float(plan["touched_rows"])
    if plan["kind"] == 0:
        return 8.0 * P * classes * P
    if plan["kind"] == 2 and np.all(U[np.abs(U) != 0] == 1):
        return 0.0
    return 6.0 * classes * rows


def circuit_method_flops(qb, circ, prec) -> float:
    return sum(method_flops(qb.qd_plan_gate(circ.dims, prec, g.wires, g.U, g.controls or None,
                                            g.values or None), g.U) for g in circ.gates)


def aggregate(units_per_rank, seconds_per_rank):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    t = max(seconds_per_rank)
    return sum(units_per_rank) / t, t


def parse_clocks(lines):
    """Summarise `nvidia-smi --query-gpu=...` CSV lines sampled during the timed region."""
    sm, smax, power, reasons = [], [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 9 or not parts[1].split()[0].isdigit():
            continue
        try:
            sm.append(float(parts[1].split()[0]))
            smax.append(float(parts[2].split()[0]))
            power.append(float(parts[3].split()[0]))
        except ValueError:
            continue
        for nm, val in zip(names, parts[5:9]):
            if val.lower() == "active":
                reasons.add(nm)
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
    loaded = [s for s, p in zip(sm, power) if p > 0.3 * max(power)] or sm
    return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
            "samples": len(sm)}


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln)

    def stop(self):
        if self.proc is None:
            return parse_clocks([])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        return parse_clocks(self.lines)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = {
    "gate": ("qd_kernels.cu", "qd_internal.cuh"),
    "fused": ("qd_fusion.cu", "qd_internal.cuh", "qd_program.h", "qd_tc_common.cuh"),
    "tc": ("qd_tc.cu", "qd_internal.cuh", "qd_tc_common.cuh"),
}
TRAFFIC_FILES = {"gate": "gate_kernel_traffic.json", "fused": "fused_kernel_traffic.json",
                 "tc": "tc_kernel_traffic.json"}


def kernel_source_hash(kind: str = "gate") -> str:
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_2410_17876_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(key: str, kind: str = "gate"):
    """DRAM bytes per launch of the kernel on the workload ``key`` from the
    committed ncu summary, if it was taken on the current kernel source
    (else None)."""
    p = os.path.join(ROOT, "profiles", TRAFFIC_FILES[kind])
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_source_hash") != kernel_source_hash(kind):
        return None
    ent = d.get(key)
    return None if ent is None else ent.get("dram_bytes_per_launch")


# ----------------------------------------------------------------------------------------------
# Distributed set-up
# ----------------------------------------------------------------------------------------------
def dist_setup(n_gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = os.environ.get("QD_BENCH_BACKEND", "nccl")
        if backend == "nccl":
            import torch

            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------------------------
# CPU oracle baseline
# ----------------------------------------------------------------------------------------------
def oracle_sample(circ, budget_s: float, nthreads: int):
    """Time the oracle on the first gates of the circuit on the full state until
    about ``budget_s`` seconds of work; returns (updates/s, gates run, seconds)."""
    import oracle

    psi = oracle.zero_state(circ.dims)
    tmp = np.empty_like(psi)
    done, upd, t0 = 0, 0, time.perf_counter()
    for g in circ.gates:
        oracle.apply_gate(circ.dims, psi, g, nthreads=nthreads, out=tmp)
        psi, tmp = tmp, psi
        done += 1
        upd += gate_updates(circ.dims, g)
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return upd / dt, done, dt


def run_reference(args):
    rank, world, _ = dist_setup(args.gpus)
    if rank != 0:
        return 0
    import oracle
    from paper_2410_17876_gb300 import inputs as gen

    oracle.build()
    pre = gen.prefix_circuit(gen.config2_circuit(), PREFIX_WIRES)
    nthreads = oracle.max_threads()
    per_step_budget = max(1.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        oracle_sample(pre, per_step_budget / 4, nthreads)
    vals, gates_run, secs = [], [], []
    for _ in range(args.steps):
        v, n, dt = oracle_sample(pre, per_step_budget, nthreads)
        vals.append(v)
        gates_run.append(n)
        secs.append(dt)
    value = statistics.median(vals)
    sample = (f"first {min(gates_run)}-{max(gates_run)} of the {len(pre.gates)} gates per step of the workload's "
              f"{PREFIX_WIRES}-wire prefix ({pre.D:,} amplitudes), FP64, {nthreads} OpenMP threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "prec": "c128 (FP64 CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------------------
LARGE_PATHS = (("per_gate", False, None), ("tile_fused", "tile", None), ("block_fused_tf32x3", "block", "tf32x3"),
               ("block_fused_bf16x3", "block", "bf16x3"), ("block_fused_fp32", "block", "fp32"))


def measure_large(qb, gen, torch, stream, amp_bytes_c64=8):
    """18 qubits + 8 qutrits (1,719,926,784 amplitudes, 13.76 GB complex64), 200 gates:
    one timed run per path -- per-gate kernels, shared-memory tile passes, and
    composed blocks of up to 64 dimensions on TF32x3 / BF16x3 tensor cores or
    FP32 CUDA cores; the per-gate kernel's HBM fraction on its dense gates.
    Each path also runs the circuit's 20-wire prefix; those outputs are kept
    (``_prefix``) for the comparison with the FP64 oracle in the CPU leg."""
    circ = gen.config2_circuit()
    upd = circuit_updates(circ)
    st = qb.State(circ.dims, prec=qb.QD_C64, stream=stream)
    out = {"workload": "18 qubits + 8 qutrits (1,719,926,784 amplitudes), 200 gates, complex64",
           "updates_per_circuit": upd}
    peak, _ = measured_peaks()
    for name, fuse, tc in LARGE_PATHS:
        kw = {"tc_mode": tc} if tc else {}
        st.reset()
        st.run(circ, fuse=fuse, **kw)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st.reset()
        e0.record(stream)
        st.run(circ, fuse=fuse, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        out[name] = {"seconds": t, "value": upd / t, "unit": UNIT}
        if fuse == "block":
            mode = qb.QD_FUSE_BLOCK
            _, _, tiles, _ = qb.qd_plan_circuit(circ.dims, qb.QD_C64, circ, mode=mode, with_flops=True)
            out[name]["passes"] = len(tiles)
    # per-launch roofline of the dense single-wire gates (uncontrolled Haar)
    dense = [g for g in circ.gates if not g.controls][:12]
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(dense) + 1)]
    evs[0].record(stream)
    for i, g in enumerate(dense):
        st.apply(g)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    tt = sum(evs[i].elapsed_time(evs[i + 1]) for i in range(len(dense))) / 1e3
    gbs = len(dense) * 2 * amp_bytes_c64 * circ.D / tt / 1e9
    out["dense_gate_kernel"] = {"achieved_gbs": gbs, "frac_of_measured_hbm": gbs / peak, "launches": len(dense)}
    st.close()
    torch.cuda.empty_cache()
    # the 20-wire prefix through every path (outputs for the oracle comparison)
    pre = gen.prefix_circuit(circ, 20)
    sp = qb.State(pre.dims, prec=qb.QD_C64, stream=stream)
    outs = {}
    for name, fuse, tc in LARGE_PATHS:
        sp.reset()
        sp.run(pre, fuse=fuse, **({"tc_mode": tc} if tc else {}))
        outs[name] = sp.raw().astype(np.complex64)
    sp.close()
    out["_prefix"] = (pre, outs)
    return out


def measure_stride_sweep(qb, gen, torch, stream, reps=20, amp_bytes=8):
    """Per-gate kernel over every wire position of the 12-qubit + 8-qutrit layout
    (complex64): a Haar dense gate, a diagonal phase gate (no unit entry) and a
    dense gate controlled by the next wire (value d_c - 1), each timed over ``reps``
    launches with CUDA events; achieved GB/s from the algorithmic bytes."""
    circ = gen.config1_circuit()
    dims = circ.dims
    rng = np.random.Generator(np.random.PCG64(20))
    st = qb.State(dims, prec=qb.QD_C64, stream=stream)
    peak, _ = measured_peaks()
    rows = []

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    for w, d in enumerate(dims):
        H = gen.haar(d, rng)
        Z = np.diag(np.exp(2j * np.pi * (np.arange(d) + 0.5) / d))
        c = (w + 1) % len(dims)
        row = {"wire": w, "d": d, "stride": int(np.prod(dims[:w], dtype=np.int64))}
        for kind, fn, touched in (
                ("dense", lambda: qb.qd_apply_gate(st.handle, w, H), circ.D),
                ("diagonal", lambda: qb.qd_apply_gate(st.handle, w, Z), circ.D),
                ("controlled", lambda: qb.qd_apply_controlled(st.handle, w, H, [c], [dims[c] - 1]),
                 circ.D // dims[c])):
            t = timed(fn)
            gbs = 2 * amp_bytes * touched / t / 1e9
            row[kind] = {"us": 1e6 * t, "gbs": gbs, "frac_of_measured_hbm": gbs / peak}
        rows.append(row)
    st.close()
    return {"workload": "12 qubits + 8 qutrits (26,873,856 amplitudes), complex64, every wire",
            "repeats": reps, "rows": rows,
            "dense_frac_min": min(r["dense"]["frac_of_measured_hbm"] for r in rows),
            "dense_frac_median": float(np.median([r["dense"]["frac_of_measured_hbm"] for r in rows]))}


def measure_sparse_ghz(qb, gen, reps=20):
    """GHZ preparation on sparse states (qd_sparse_run: one launch per circuit, the
    non-zero amplitudes in one CTA's shared memory), at the sizes of the paper's
    sparse runs (62 qubits, 39 qutrits, 31 ququads, 27 ququints: 0.15 / 0.188 / 0.2 /
    0.21 ms on its CPU) and beyond 64-bit indices.  Wall time of the synchronous call
    (gate upload, kernel, status read-back), median of ``reps``; the result is checked
    against the closed form sum_k |k...k> / sqrt(d)."""
    paper_ms = {(2, 62): 0.15, (3, 39): 0.188, (4, 31): 0.2, (5, 27): 0.21}
    rows = []
    for d, n in ((2, 62), (3, 39), (4, 31), (5, 27), (2, 127), (3, 64), (5, 42)):
        dims = (d,) * n
        circ = gen.ghz_circuit(dims)
        qb.circuit_arrays(circ)
        ts = []
        ok = True
        for _ in range(reps + 2):
            s = qb.qd_sparse_create(dims)
            t0 = time.perf_counter()
            qb.qd_sparse_run(s, circ)
            ts.append(time.perf_counter() - t0)
            got = qb.qd_sparse_get(s)
            qb.qd_sparse_destroy(s)
            stride_sum = sum(d ** w for w in range(n))
            ok = ok and len(got) == d and all(abs(got.get(k * stride_sum, 0) - d ** -0.5) < 1e-15 for k in range(d))
        t = float(np.median(ts[2:]))
        row = {"d": d, "wires": n, "gates": len(circ.gates), "ms": 1e3 * t, "closed_form_ok": ok}
        if (d, n) in paper_ms:
            row["paper_ms_cpu"] = paper_ms[(d, n)]
        rows.append(row)
    return {"workload": "GHZ circuits on sparse states (F_d on wire 0, then controlled X_{+v} on every other "
                        "wire), complex128", "rows": rows}


def measure_sparse_grid(qb, gen, reps=5):
    """A sparse state beyond the one-CTA buffers (qd_sparse_reserve, grid tier):
    Fourier gates on 12 of 16 wires, then 40 seeded single-wire gates (Haar,
    shifts and phases, 40% controlled).  Wall time of the synchronous
    qd_sparse_run, median of ``reps``."""
    rng = np.random.Generator(np.random.PCG64(971))
    dims = (2, 3, 2, 2, 3, 2, 2, 2, 3, 2, 2, 2, 2, 3, 2, 2)
    gates = [gen.Gate((w,), gen.fourier(dims[w])) for w in range(0, 12)]
    for _ in range(40):
        t = int(rng.integers(0, len(dims)))
        d = dims[t]
        k = rng.random()
        U = gen.haar(d, rng) if k < 0.2 else (gen.x_plus(d, 1) if k < 0.6 else gen.z_gen(d))
        c = int(rng.integers(0, len(dims)))
        if rng.random() < 0.4 and c != t:
            gates.append(gen.Gate((t,), U, (c,), (int(rng.integers(0, dims[c])),)))
        else:
            gates.append(gen.Gate((t,), U))
    circ = gen.Circuit(dims, gates)
    ts, nnz = [], 0
    for _ in range(reps + 1):
        s = qb.qd_sparse_create(dims)
        qb.qd_sparse_reserve(s, 1 << 18)
        n0 = qb.qd_launch_count()
        t0 = time.perf_counter()
        qb.qd_sparse_run(s, circ)
        ts.append(time.perf_counter() - t0)
        launches = qb.qd_launch_count() - n0
        nnz = qb.qd_sparse_nnz(s)
        qb.qd_sparse_destroy(s)
    return {"workload": "16 wires (12 qubits, 4 qutrits), 52 single-wire gates, complex128 sparse state",
            "gates": len(circ.gates), "nnz": nnz, "ms": 1e3 * float(np.median(ts[1:])), "launches": launches}


def measure_tile_costs(qb, gen, torch, stream, reps=5):
    """Marginal cost of one gate or composed block inside a shared-memory tile pass
    on the 12-qubit + 8-qutrit layout (complex64): the pass with N + 6 copies minus
    the pass with N, over 6 (N = 2), timed with CUDA events through
    qd_apply_circuit.  Single gates use block_dim 1 (no composition); blocks are
    runs of gates on 2-4 wires composed in binary64, consecutive blocks sharing a
    wire so that they neither commute nor merge.  The pass floor is the cost of a
    pass holding two phase gates."""
    circ = gen.config1_circuit()
    dims = circ.dims
    rng = np.random.Generator(np.random.PCG64(21))
    qub = [i for i, d in enumerate(dims) if d == 2]
    qut = [i for i, d in enumerate(dims) if d == 3]
    st = qb.State(dims, prec=qb.QD_C64, stream=stream)

    def timed(gates, bd):
        c = gen.Circuit(dims, gates)
        st.run(c, fuse="tile", block_dim=bd)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            st.run(c, fuse="tile", block_dim=bd)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    def block(ws):
        g = [gen.Gate((w,), gen.haar(dims[w], rng)) for w in ws]
        return g + [gen.Gate((ws[i + 1],), gen.haar(dims[ws[i + 1]], rng), (ws[i],), (1,)) for i in range(len(ws) - 1)]

    kinds = {
        "qubit_gate": (lambda i: [gen.Gate((qub[2 + i % 2],), gen.haar(2, rng))], 1, 16),
        "qutrit_gate": (lambda i: [gen.Gate((qut[2 + i % 2],), gen.haar(3, rng))], 1, 24),
        "qubit_phase_gate": (lambda i: [gen.Gate((qub[2 + i % 2],), np.diag(np.exp(1j * rng.random(2))))], 1, 6),
        "qutrit_shift_gate": (lambda i: [gen.Gate((qut[2 + i % 2],), gen.x_plus(3, 1))], 1, 24),
        "block_9_two_qutrits": (lambda i: block(qut[0:2] if i % 2 == 0 else qut[1:3]), 9, 72),
        "block_16_four_qubits": (lambda i: block(qub[0:4] if i % 2 == 0 else qub[3:7]), 16, 128),
    }
    out = {"workload": "12 qubits + 8 qutrits (26,873,856 amplitudes), complex64, one tile pass",
           "alu_peak_tflops": FP32_TFLOPS, "rows": {}}
    Z = np.diag([1, -1]).astype(complex)
    out["pass_floor_us"] = 1e6 * timed([gen.Gate((qub[-1],), Z), gen.Gate((qub[-2],), Z)], 1)
    for name, (mk, bd, flop_per_amp) in kinds.items():
        base = sum((mk(i) for i in range(2)), [])
        more = sum((mk(i) for i in range(8)), [])
        t = (timed(more, bd) - timed(base, bd)) / 6
        out["rows"][name] = {"us": 1e6 * t, "flop_per_amp": flop_per_amp,
                             "tflops": flop_per_amp * circ.D / t / 1e12 if t > 0 else None}
    st.close()
    return out


def measure_lazy(qb, gen, torch, stream):
    """The benchmark circuit applied gate by gate through the C ABI (qd_apply_gate /
    qd_apply_controlled), complex64, without and with the lazy frame (qd_set_lazy:
    single-wire phase and permutation gates folded into a per-wire relabeling and
    phase vector, no launch).  CUDA events around the 500 calls plus, with the frame,
    the final materialisation (qd_set_lazy(st, 0))."""
    circ = gen.config1_circuit()
    st = qb.State(circ.dims, prec=qb.QD_C64, stream=stream)
    out = {"workload": "12 qubits + 8 qutrits (26,873,856 amplitudes), 500 gates, complex64, one call per gate"}
    for name, lazy in (("eager", False), ("lazy", True)):
        for rep in range(2):  # the first run warms up
            st.reset()
            torch.cuda.synchronize()
            n0 = qb.qd_launch_count()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if lazy:
                st.set_lazy(True)
            st.run_gate_by_gate(circ)
            if lazy:
                st.set_lazy(False)
            e1.record(stream)
            torch.cuda.synchronize()
        out[name] = {"ms": e0.elapsed_time(e1), "launches": qb.qd_launch_count() - n0,
                     "updates_per_s": circuit_updates(circ) / (e0.elapsed_time(e1) / 1e3)}
    st.close()
    return out


def measure_many_controls(qb, gen, torch, stream, reps=10):
    """Controlled X_{+1} with M = 1..16 controls on the 12-qubit + 8-qutrit layout
    (26,873,856 complex64 amplitudes): the digit-insertion enumeration
    (qd_apply_controlled, only matching classes visited) against the paper's
    scanning formulation (qd_apply_controlled_scan, every target class visited and
    its M control digits tested).  Controls: the highest wires other than the
    target, values drawn from a fixed seed."""
    circ = gen.config1_circuit()
    dims = circ.dims
    rng = np.random.Generator(np.random.PCG64(16))
    target = [w for w, d in enumerate(dims) if d == 2][0]
    others = sorted((w for w in range(len(dims)) if w != target), reverse=True)
    st = qb.State(dims, prec=qb.QD_C64, stream=stream)
    X = gen.x_plus(2, 1)
    out = {"workload": "12 qubits + 8 qutrits (26,873,856 amplitudes), complex64, controlled X_{+1} on wire "
                       f"{target}", "rows": []}

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    for m in (1, 2, 4, 8, 12, 16):
        cw = others[:m]
        cv = [int(rng.integers(0, dims[w])) for w in cw]
        t_enum = timed(lambda: qb.qd_apply_controlled(st.handle, target, X, cw, cv))
        t_scan = timed(lambda: qb.qd_apply_controlled_scan(st.handle, target, X, cw, cv))
        matched = circ.D // 2 // int(np.prod([dims[w] for w in cw]))
        out["rows"].append({"controls": m, "matching_classes": matched, "enumeration_us": 1e6 * t_enum,
                            "scan_us": 1e6 * t_scan, "scan_over_enumeration": t_scan / t_enum})
    st.close()
    return out


def measure_batched(qb, gen, torch, stream, reps=3):
    """8192 independent circuits (widths 4-12, dims {2,3,4,5}, depths 20-300),
    complex64, captured in a CUDA graph, through each path of the larger
    circuits: the device-side layer queue (one launch per pass position for
    all of them) and one program per circuit on auxiliary streams.  Build
    and first run: wall time; relaunches: CUDA events."""
    t0 = time.perf_counter()
    circs = gen.config3_batch()
    t_gen = time.perf_counter() - t0
    upd = sum(circuit_updates(c) for c in circs)
    out = {"workload": "8192 circuits, widths 4-12, dims {2,3,4,5}, depths 20-300, complex64", "generate_s": t_gen}
    for name, path in (("layer_queue", qb.QD_BATCH_LAYERS), ("stream_programs", qb.QD_BATCH_STREAMS)):
        b = qb.qd_batch_create(qb.QD_C64, stream.cuda_stream)
        t0 = time.perf_counter()
        n0 = qb.qd_launch_count()
        qb.qd_batch_run(b, circs, use_graph=True, path=path)
        qb.qd_batch_synchronize(b)
        t_first = time.perf_counter() - t0
        launches = qb.qd_launch_count() - n0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            qb.qd_batch_relaunch(b)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / reps
        norms = qb.qd_batch_norms(b, len(circs))
        qb.qd_batch_destroy(b)
        out[name] = {"circuits_per_s": len(circs) / t, "value": upd / t, "unit": UNIT, "seconds_per_batch": t,
                     "first_run_wall_s": t_first, "launches_per_batch": launches,
                     "max_norm_error": float(np.max(np.abs(norms - 1.0)))}
        torch.cuda.empty_cache()
    best = max(("layer_queue", "stream_programs"), key=lambda k: out[k]["circuits_per_s"])
    out.update(circuits_per_s=out[best]["circuits_per_s"], value=out[best]["value"], unit=UNIT, best_path=best)
    return out


def measure_serving(qb, gen, torch, trace, plain_budget_s=6.0, capacity_s=2.0, in_flight=(16, 64, 256, 1024)):
    """Serving the Poisson trace (mean 2000 arrivals/s for 10 s, widths 4-16,
    dims {2,3,4}, 16 <= D <= 1.6e7, depths 50-500; complex64 states, FP64
    norms):
      * open loop: every request submitted ahead with its arrival time on the
        server clock; p50/p99 latency = done - arrival;
      * closed loop (capacity): N requests kept in flight (a new one submitted
        as each finishes, the trace's circuits in order) for ``capacity_s``
        seconds, for each N in ``in_flight``; circuits/s and p50/p99 of
        done - submit;
      * the plain path: complex128, one circuit at a time, one kernel per
        gate, state created and destroyed per request, for about
        ``plain_budget_s`` seconds on the trace's circuits in order;
      * served_over_plain = the best closed-loop circuits/s over the plain
        path's circuits/s.
    1% of the open-loop requests (a seeded draw over all sizes) keep their
    states (``_sample``) for the comparison with the FP64 oracle in the CPU leg."""
    circs = [c for _, c in trace]
    arr = np.array([t for t, _ in trace])
    duration = float(np.ceil(arr.max())) if len(arr) else 0.0
    upd = np.array([circuit_updates(c) for c in circs], dtype=np.float64)
    for c in circs:
        qb.circuit_arrays(c)
    rng = np.random.Generator(np.random.PCG64(44))
    sample = sorted(int(i) for i in rng.permutation(len(circs))[:max(1, len(circs) // 100)])
    keep = set(sample)
    srv = qb.qd_server_create(qb.QD_C64, hbm_budget_bytes=48 << 30, max_slots=32)
    base = qb.qd_server_now(srv) + 1.0 + 4e-4 * len(circs)
    ids = [qb.qd_server_submit_at(srv, c, base + float(t), keep_state=(i in keep)) for i, (c, t) in
           enumerate(zip(circs, arr))]
    late = qb.qd_server_now(srv) > base
    qb.qd_server_drain(srv, 600)
    res = {}
    while len(res) < len(ids):
        for r in qb.qd_server_poll(srv):
            res[r["id"]] = r
    lat = np.array([res[i]["t_done"] - res[i]["t_arrival"] for i in ids])
    done = np.array([res[i]["t_done"] for i in ids])
    ok = all(res[i]["status"] == 0 for i in ids)
    span = float(done.max() - (base + arr.min()))
    # the sampled requests' results, compared with the FP64 oracle in the CPU leg (smallest first)
    kept = sorted(((circs[i], qb.qd_server_get_amplitudes(srv, ids[i], circs[i].D).astype(np.complex64))
                   for i in sample), key=lambda x: x[0].D)
    for i in sample:
        qb.qd_server_release(srv, ids[i])
    # closed loop: N requests in flight
    capacity = []
    k = 0
    for n in in_flight:
        sub = {}
        t_end = time.perf_counter() + capacity_s
        for _ in range(n):
            sub[qb.qd_server_submit(srv, circs[k % len(circs)])] = k % len(circs)
            k += 1
        finished, lats, upd_done = 0, [], 0.0
        t0 = qb.qd_server_now(srv)
        while time.perf_counter() < t_end:
            rs = qb.qd_server_poll(srv)
            if not rs:
                time.sleep(2e-4)
            for r in rs:
                ci = sub.pop(r["id"])
                finished += 1
                upd_done += upd[ci]
                lats.append(r["t_done"] - r["t_arrival"])
                sub[qb.qd_server_submit(srv, circs[k % len(circs)])] = k % len(circs)
                k += 1
        t1 = qb.qd_server_now(srv)
        qb.qd_server_drain(srv, 600)
        while sub:
            for r in qb.qd_server_poll(srv):
                sub.pop(r["id"], None)
        capacity.append({"in_flight": n, "circuits_per_s": finished / (t1 - t0),
                         "updates_per_s": upd_done / (t1 - t0),
                         "p50_latency_s": float(np.percentile(lats, 50)) if lats else None,
                         "p99_latency_s": float(np.percentile(lats, 99)) if lats else None,
                         "finished": finished, "seconds": t1 - t0})
    qb.qd_server_destroy(srv)
    # plain path: complex128, one circuit at a time, one kernel per gate
    n_plain, t_plain = 0, 0.0
    t0 = time.perf_counter()
    for c in circs:
        h = qb.qd_state_create(c.dims, qb.QD_C128)
        qb.qd_apply_circuit(h, c, qb.QD_FUSE_OFF)
        qb.qd_norm(h)
        qb.qd_state_destroy(h)
        n_plain += 1
        t_plain = time.perf_counter() - t0
        if t_plain > plain_budget_s:
            break
    plain_cps = n_plain / t_plain
    best = max(capacity, key=lambda r: r["circuits_per_s"])
    return {"workload": f"Poisson arrivals at 2000/s for {duration:g} s ({len(circs)} requests), widths 4-16, "
                        "dims {2,3,4}, 16 <= D <= 1.6e7, depths 50-500, complex64 with FP64 norms",
            "open_loop": {"circuits_per_s": len(circs) / span, "p50_latency_s": float(np.percentile(lat, 50)),
                          "p99_latency_s": float(np.percentile(lat, 99)),
                          "offered_updates_per_s": float(upd.sum() / duration),
                          "served_updates_per_s": float(upd.sum() / span), "all_ok": ok,
                          "submission_late": bool(late)},
            "closed_loop": capacity,
            "capacity_circuits_per_s": best["circuits_per_s"],
            "_sample": kept,
            "plain_c128_one_at_a_time": {"circuits_per_s": plain_cps, "requests_timed": n_plain,
                                         "seconds": t_plain},
            "served_over_plain": best["circuits_per_s"] / plain_cps,
            "served_over_plain_basis": "closed-loop capacity (best N) over the plain path, same circuits in order"}


def oracle_checks(extra, nthreads: int, budget_s: float = 60.0) -> dict:
    """CPU leg: the FP64 oracle on what the GPU measurements kept -- the large
    workload's 20-wire prefix (every path's error) and the 1% serving sample
    (until ``budget_s`` is spent).  Fills the reports in ``extra`` in place."""
    import oracle

    def errs(ref, got):
        got = np.asarray(got, dtype=np.complex128)
        ov = np.vdot(ref, got)
        inf = float(1 - abs(ov) ** 2 / (np.vdot(ref, ref).real * np.vdot(got, got).real))
        return float(np.max(np.abs(got - ref))), inf

    t0 = time.perf_counter()
    if "large_state_paths" in extra:
        pre, outs = extra["large_state_paths"].pop("_prefix")
        ref = oracle.run_circuit(pre, nthreads=nthreads)
        rep = {"prefix": f"lowest 20 wires ({pre.D} amplitudes), {len(pre.gates)} gates"}
        for name, got in outs.items():
            e, inf = errs(ref, got)
            g64 = np.asarray(got, dtype=np.complex128)
            rep[name] = {"max_abs_err": e, "infidelity": inf, "norm_minus_1": float(np.vdot(g64, g64).real - 1.0)}
        extra["large_state_paths"]["error_vs_fp64_oracle"] = rep
    if "serving" in extra:
        kept = extra["serving"].pop("_sample")
        es, infs, big = [], [], 0
        for c, got in kept:  # smallest first, until the budget is spent
            if time.perf_counter() - t0 > budget_s:
                break
            e, inf = errs(oracle.run_circuit(c, nthreads=nthreads), got)
            es.append(e)
            infs.append(inf)
            big += c.D > (1 << 20)
        extra["serving"]["oracle_sample"] = {
            "requests": len(es), "of_sampled": len(kept), "above_2^20_amplitudes": big,
            "sampled_above_2^20": sum(1 for c, _ in kept if c.D > (1 << 20)),
            "max_abs_err": max(es) if es else None, "max_infidelity": max(infs) if infs else None,
            "rule": "a seeded 1% of all requests, checked smallest first within the CPU leg's time budget"}
    return {"seconds": time.perf_counter() - t0}


def pass_attribution(qb, gen, torch, st, circ, prec, fuse, fopts, stream, amp_bytes):
    """One extra, untimed run of the circuit with CUDA events around every
    pass of its execution plan (one qd_apply_circuit call per pass), each
    pass attributed to the kernel family that runs it.  Per family: seconds,
    passes, HBM bytes of a pass (2 s D for tile and tensor-core passes, the
    algorithmic bytes of the gate otherwise), the method's own flops of the
    gates it applies (``method_flops``), the composed-block flops the
    planner reports, and the MMA flops of tensor-core passes."""
    D = circ.D
    if fuse:
        mode = {"tile": qb.QD_FUSE_TILE, "block": qb.QD_FUSE_BLOCK}[fuse]
        popts = {k: v for k, v in fopts.items() if k != "tc_mode"}  # the plan does not depend on it
        order, pass_of, tiles, pflops = qb.qd_plan_circuit(circ.dims, prec, circ, mode=mode, with_flops=True,
                                                           **popts)
        groups = [[] for _ in range(len(tiles))]
        for g_idx, p_idx in zip(order, pass_of):
            groups[p_idx].append(circ.gates[g_idx])
    else:
        groups = [[g] for g in circ.gates]
        tiles, pflops = [0] * len(groups), [0.0] * len(groups)
    subs = [gen.Circuit(circ.dims, gl) for gl in groups]
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(subs) + 1)]
    st.reset()
    torch.cuda.synchronize()
    evs[0].record(stream)
    for i, sc in enumerate(subs):
        st.run(sc, fuse=fuse, **fopts)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    fam = {}
    for i, gl in enumerate(groups):
        t = evs[i].elapsed_time(evs[i + 1]) / 1e3
        plans = [qb.qd_plan_gate(circ.dims, prec, g.wires, g.U, g.controls or None, g.values or None) for g in gl]
        wires = set()
        for g in gl:
            wires |= set(g.wires) | set(g.controls)
        P = int(np.prod([circ.dims[w] for w in wires]))
        if fuse and tiles[i] > 0:
            k, nbytes = "tile", 2 * amp_bytes * D
        elif fuse and len(gl) > 1 and prec == qb.QD_C64 and fopts.get("tc_mode") == "bf16x3" and P >= 9:
            # BF16x3 composed blocks (no controls) of 9..64 dimensions stream through the tile ring
            k, nbytes = "ring", 2 * amp_bytes * D
        elif fuse and len(gl) > 1 and prec == qb.QD_C64 and P >= 17:
            k, nbytes = "tc", 2 * amp_bytes * D
        elif len(gl) == 1:
            k, nbytes = "gate", algorithmic_bytes(plans[0], amp_bytes)
        else:
            k, nbytes = "gate", 2 * amp_bytes * D
        f = fam.setdefault(k, {"time": 0.0, "bytes": 0, "composed_flops": 0.0, "method_flops": 0.0, "n": 0,
                               "mma_flops": 0.0, "gates": 0})
        f["time"] += t
        f["bytes"] += nbytes
        f["composed_flops"] += float(pflops[i])
        f["method_flops"] += sum(method_flops(pl, g.U) for pl, g in zip(plans, gl))
        f["n"] += 1
        f["gates"] += len(gl)
        if k == "tc":  # 3 products x 16 k-steps of M=128, N=64, K=8 per 64 classes
            f["mma_flops"] += math.ceil(D / P / 64) * 48 * 2 * 128 * 64 * 8
        elif k == "ring":  # useful products: 3 x 2 (2P)^2 per class, D / P classes
            f["mma_flops"] += 24.0 * P * D
    return fam


KERNEL_NAMES = {"tile": "k_fused_tile (shared-memory tile pass)",
                "tc": "k_block_tc (tcgen05 tensor-core block pass, TF32x3)",
                "ring": "k_block_tc_ring (tcgen05 block pass over a ring of bulk-copied tiles, BF16x3)",
                "gate": "k_gate1 / k_gate_tile (per-gate passes)"}


def roofline_of(fam, traffic_key, is_c64):
    """Roofline record of the family with the most time (see ``pass_attribution``);
    ``traffic_key``: the workload's entry in the committed ncu traffic summaries."""
    dom = max(fam, key=lambda k: fam[k]["time"])
    f = fam[dom]
    peak, peak_kind = measured_peaks()
    t = f["time"]
    if dom == "tile":
        alu_peak = FP32_TFLOPS if is_c64 else FP64_TFLOPS
        roof = {"kernel": KERNEL_NAMES[dom], "bound": "alu", "achieved": f["method_flops"] / t / 1e12,
                "peak": alu_peak, "unit": "TFLOP/s",
                "work": "the method's own flops of the pass's gates: 8 P per amplitude of every visited class for "
                        "dense P x P gates, 6 per changed amplitude for phases, 0 for pure permutations",
                "peak_source": "derived: " + ALU_PEAK_NOTE,
                "traffic": ncu_traffic(traffic_key, "fused"), "launches_measured": f["n"],
                "hbm_view": {"achieved_gbs": f["bytes"] / t / 1e9, "peak_gbs": peak, "frac": f["bytes"] / t / 1e9 / peak,
                             "bytes": "2 s D per pass", "peak_source": peak_kind},
                "composed_flops": {"achieved_tflops": f["composed_flops"] / t / 1e12,
                                   "frac": f["composed_flops"] / t / 1e12 / alu_peak,
                                   "work": "8 P flops per amplitude per composed P x P block (dense equivalent)"}}
        roof["frac"] = roof["achieved"] / roof["peak"]
    else:
        achieved = f["bytes"] / t / 1e9
        roof = {"kernel": KERNEL_NAMES[dom], "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": ncu_traffic(traffic_key, "tc" if dom in ("tc", "ring") else "gate"),
                "launches_measured": f["n"], "method_tflops": f["method_flops"] / t / 1e12}
        if dom == "ring":
            roof["tensor_view"] = {"achieved_tflops": f["mma_flops"] / t / 1e12, "peak_tflops": bf16_peak(),
                                   "frac": f["mma_flops"] / t / 1e12 / bf16_peak(),
                                   "work": "the three BF16 products of each class's real 2P x 2P embedding",
                                   "peak_source": "measured bf16 burst"}
        if dom == "tc":
            tf32 = tf32_peak()
            roof["tensor_view"] = {"achieved_tflops": f["mma_flops"] / t / 1e12, "peak_tflops": tf32,
                                   "frac": f["mma_flops"] / t / 1e12 / tf32,
                                   "peak_source": "measured bf16 burst x 0.489 (nominal TF32/BF16 dense ratio)"}
    roof["passes_by_kernel"] = {k: {"seconds": v["time"], "passes": v["n"], "gates": v["gates"]}
                                for k, v in fam.items()}
    return roof


def host_mem_available() -> int:
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return 0


def measure_benchmark_circuit(qb, gen, torch, stream, steps=10):
    """The 12-qubit + 8-qutrit Clifford+T-like circuit (26,873,856 amplitudes,
    500 gates): complex64 with autotuned fusion, complex128 per gate and in
    tile passes.  Each: ``steps`` timed steps (reset, circuit, norm) with CUDA
    events after a warm-up step, and the dominant kernel's roofline."""
    from paper_2410_17876_gb300 import autotune

    circ = gen.config1_circuit()
    upd = circuit_updates(circ)
    out = {"workload": BENCH_CIRCUIT, "updates_per_circuit": upd}
    for name, prec, fuse in (("c64", qb.QD_C64, "auto"), ("c128_per_gate", qb.QD_C128, False),
                             ("c128_tile", qb.QD_C128, "tile")):
        st = qb.State(circ.dims, prec=prec, stream=stream)
        fopts = {}
        if fuse == "auto":
            tuned = autotune.tune_circuit(st, circ)
            fuse = tuned["mode"] if tuned["mode"] != "off" else False
            fopts = {"max_tile_amps": tuned["max_tile_amps"], "block_dim": tuned["block_dim"],
                     "tc_mode": tuned["tc_mode"]} if fuse else {}

        def step():
            st.reset()
            st.run(circ, fuse=fuse, **fopts)
            return st.norm()

        step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3 / steps
        amp_bytes = 8 if prec == qb.QD_C64 else 16
        fam = pass_attribution(qb, gen, torch, st, circ, prec, fuse, fopts, stream, amp_bytes)
        out[name] = {"ms_per_step": 1e3 * t, "value": upd / t, "unit": UNIT, "fusion": fuse or "off",
                     "fusion_opts": fopts,
                     "roofline": roofline_of(fam, "benchmark_" + ("c64" if prec == qb.QD_C64 else "c128"),
                                             prec == qb.QD_C64)}
        st.close()
        torch.cuda.empty_cache()
    return out


def run_gpu(args):
    import torch

    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    import __graft_entry__

    if rank == 0 or world == 1:
        __graft_entry__.build()
    barrier(world)
    from paper_2410_17876_gb300 import autotune
    from paper_2410_17876_gb300 import binding as qb
    from paper_2410_17876_gb300 import inputs as gen

    trace_box = []
    trace_thread = None
    if not args.no_extra:  # the serving trace (~20k circuits) is generated while the GPU works
        trace_thread = threading.Thread(target=lambda: trace_box.append(gen.config4_trace(duration=10.0)),
                                        daemon=True)
        trace_thread.start()
    prec = qb.QD_C64
    amp_bytes = 8
    circ = gen.config2_circuit()
    upd = circuit_updates(circ)
    stream = torch.cuda.current_stream(local)
    st = qb.State(circ.dims, prec=prec, stream=stream, device=local)

    tuned = None
    if args.fuse == "auto":
        tuned = autotune.tune_circuit(st, circ, budget_s=45.0)
        fuse = tuned["mode"] if tuned["mode"] != "off" else False
        fopts = {"max_tile_amps": tuned["max_tile_amps"], "block_dim": tuned["block_dim"],
                 "tc_mode": tuned["tc_mode"]} if fuse else {}
    else:
        fuse = args.fuse if args.fuse != "off" else False
        fopts = {"max_tile_amps": args.tile} if fuse == "tile" and args.tile else {}
        if fuse and args.block_dim:
            fopts["block_dim"] = args.block_dim
        if fuse:
            fopts["tc_mode"] = args.tc_mode

    def step():
        st.reset()
        st.run(circ, fuse=fuse, **fopts)
        return st.norm()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # ---- timed region: device time with CUDA events on the launching stream ----
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    n0 = qb.qd_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = qb.qd_launch_count() - n0
    dev_s = ev0.elapsed_time(ev1) / 1e3
    barrier(world)
    clocks = sampler.stop() if sampler else None
    t_max = max_over_ranks(dev_s, world)
    value, _ = aggregate([upd * args.steps] * world, [t_max] * world)

    # ---- per-pass durations of the dominant kernel (one extra, untimed step) ----
    fam = pass_attribution(qb, gen, torch, st, circ, prec, fuse, fopts, stream, amp_bytes)
    roof = roofline_of(fam, "large_c64", True)
    step_method_flops = sum(v["method_flops"] for v in fam.values())

    # ---- end to end through the public API with host buffers ----
    # Every step is a new circuit of the workload's shape (fresh Haar
    # matrices, so the library plans, composes and uploads it: no cached
    # program), its norm read on the host and the whole final state copied
    # into pinned host memory.  With room for two pinned buffers, two states
    # on two streams alternate, so one step's read-back runs while the next
    # step computes; the clock stops when the last read-back has landed.
    # The serving trace's generation (host threads) ends first, so that the
    # host is otherwise idle during these steps.
    if trace_thread is not None:
        trace_thread.join()
    state_bytes = circ.D * amp_bytes
    e2e = None
    e2e_steps = max(4, min(args.steps, 10))
    e2e_circs = [gen.redraw_haar(circ, 1000 + i) for i in range(e2e_steps + 1)]
    assert all(circuit_updates(c) == upd for c in e2e_circs)
    h2d = sum(g.U.size * 16 + 8 * len(g.controls) for g in circ.gates)
    avail = host_mem_available()
    nbuf = 2 if avail > 4.5 * state_bytes else 1 if avail > 2.5 * state_bytes else 0
    if nbuf:
        pinned = [torch.empty(circ.D, dtype=torch.complex64, pin_memory=True) for _ in range(nbuf)]
        outs = [p.numpy() for p in pinned]
        states = [st] + [qb.State(circ.dims, prec=prec, stream=torch.cuda.Stream(local), device=local)
                         for _ in range(nbuf - 1)]
        for s_, o_ in zip(states, outs):  # warm: the second state's first run, each buffer's pages
            s_.reset()
            s_.run(e2e_circs[-1], fuse=fuse, **fopts)
            qb.qd_state_get_raw(s_.handle, o_)
        barrier(world)
        starts, norms = [], []
        up0 = qb.qd_bytes_uploaded()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            s_, o_ = states[i % nbuf], outs[i % nbuf]
            starts.append(time.perf_counter())
            # Stream order puts the reset after this state's previous
            # read-back, and the norm's host read returns only after both
            # (no host wait on the other stream's copy before the launches).
            s_.reset()
            s_.run(e2e_circs[i], fuse=fuse, **fopts)
            norms.append(s_.norm())
            qb.qd_state_get_raw_async(s_.handle, o_)
        for s_ in states:
            s_.synchronize()
        total = time.perf_counter() - t0
        uploaded = (qb.qd_bytes_uploaded() - up0) // e2e_steps
        last = (e2e_steps - 1) % nbuf
        head = states[last].buf[:2000].cpu().numpy().view(np.complex64)
        readback_ok = bool(np.array_equal(outs[last][:1000], head))
        e2e_s = max_over_ranks(total / e2e_steps, world)
        e2e = {"value": world * upd / e2e_s, "unit": UNIT, "h2d_bytes_per_step": uploaded,
               "gate_input_bytes_per_step": h2d,
               "d2h_bytes_per_step": outs[0].nbytes + 8, "steps": e2e_steps, "ms_per_step": 1e3 * e2e_s,
               "ms_total": 1e3 * total,
               "ms_between_step_starts": [round(1e3 * (b - a), 1) for a, b in zip(starts, starts[1:])],
               "pipelined": nbuf == 2, "max_norm_error": max(abs(x - 1.0) for x in norms),
               "readback_matches_device": readback_ok, "host_mem_available_gb": round(avail / 1e9, 1),
               "what": "every step a new circuit of the workload's shape (fresh Haar matrices from host "
                       "memory: planned, composed and uploaded by qd_apply_circuit), the norm read on the "
                       "host, and the whole final state copied into pinned host memory (qd_state_get_raw_async); "
                       "h2d_bytes_per_step: the descriptors, composed block matrices and tensor-core operands the "
                       "library uploaded (qd_bytes_uploaded), built from gate_input_bytes_per_step of gate records"
                       + ("; two states on two streams alternate, so a step's read-back overlaps the next "
                          "step's compute; time from the first step's start to the last read-back's end"
                          if nbuf == 2 else "; one state, steps back to back")}
        for s_ in states[1:]:
            s_.close()
        del pinned, outs, states, s_
    st.close()
    del st
    torch.cuda.empty_cache()

    # ---- the other workloads of the path, each one timed run (rank 0 reports its own) ----
    extra = {}
    if not args.no_extra:
        extra["benchmark_circuit"] = measure_benchmark_circuit(qb, gen, torch, stream)
        torch.cuda.empty_cache()
        extra["large_state_paths"] = measure_large(qb, gen, torch, stream, amp_bytes_c64=8)
        torch.cuda.empty_cache()
        extra["stride_sweep"] = measure_stride_sweep(qb, gen, torch, stream)
        torch.cuda.empty_cache()
        extra["many_controls"] = measure_many_controls(qb, gen, torch, stream)
        extra["sparse_ghz"] = measure_sparse_ghz(qb, gen)
        try:
            extra["sparse_grid"] = measure_sparse_grid(qb, gen)
        except Exception as e:  # reported, never fatal to the bench line
            extra["sparse_grid"] = {"error": str(e)[:200]}
        torch.cuda.empty_cache()
        extra["lazy_frame"] = measure_lazy(qb, gen, torch, stream)
        extra["tile_costs"] = measure_tile_costs(qb, gen, torch, stream)
        torch.cuda.empty_cache()
        extra["batched"] = measure_batched(qb, gen, torch, stream)
        torch.cuda.empty_cache()
        extra["serving"] = measure_serving(qb, gen, torch, trace_box[0])
        torch.cuda.empty_cache()

    # ---- CPU oracle baseline (rank 0, N = 1 only): the workload's 20-wire prefix ----
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        nthreads = oracle.max_threads()
        pre = gen.prefix_circuit(circ, PREFIX_WIRES)
        v, n, dt = oracle_sample(pre, args.cpu_seconds, nthreads)
        cpu = {"value": v, "unit": UNIT, "cores": nthreads, "kind": "oracle",
               "sample": f"first {n} of the {len(pre.gates)} gates of the workload's {PREFIX_WIRES}-wire prefix "
                         f"({pre.D:,} amplitudes; the gates whose wires all lie in it), FP64, {dt:.1f} s"}
        if extra:
            cpu["checks"] = oracle_checks(extra, nthreads)
    for rep in extra.values():  # outputs kept for checks that did not run
        for k in [k for k in rep if k.startswith("_")]:
            rep.pop(k)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "prec": "c64", "fusion": fuse or "off",
                       "fusion_opts": fopts, "autotuned": tuned is not None,
                       "autotune_table_s": tuned.get("table") if tuned else None,
                       "amplitudes": circ.D, "gates": len(circ.gates), "state_bytes": state_bytes,
                       "l2": f"state {state_bytes / 1e9:.2f} GB > {L2_BYTES / 1e6:.0f} MB L2, no flush",
                       "parallelism": f"replicas x{world}"},
            "method_tflops": step_method_flops * args.steps / t_max / 1e12,
            "per_gate_equivalent_gbs": sum(algorithmic_bytes(qb.qd_plan_gate(circ.dims, prec, g.wires, g.U,
                                                                             g.controls or None,
                                                                             g.values or None), amp_bytes)
                                           for g in circ.gates) * args.steps / t_max / 1e9,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def run_ncu_case(args):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2410_17876_gb300 import binding as qb
    from paper_2410_17876_gb300 import inputs as gen

    prec = qb.QD_C64 if args.prec == "c64" else qb.QD_C128
    circ = gen.config1_circuit()
    rng = np.random.Generator(np.random.PCG64(99))
    st = qb.State(circ.dims, prec=prec)
    for w in (0, 5, 10, 15, 19, 3):
        st.apply(gen.Gate((w,), gen.haar(circ.dims[w], rng)))
    st.synchronize()
    st.close()
    torch.cuda.synchronize()
    return 0


def run_ncu_fused_case(args):
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2410_17876_gb300 import binding as qb
    from paper_2410_17876_gb300 import inputs as gen

    prec = qb.QD_C64 if args.prec == "c64" else qb.QD_C128
    if args.ncu_workload == "prefix":
        circ = gen.prefix_circuit(gen.config2_circuit(), PREFIX_WIRES)
    else:
        circ = gen.config1_circuit()
    st = qb.State(circ.dims, prec=prec)
    fuse = "tile" if args.fuse in ("auto", "tile") else args.fuse
    opts = {"max_tile_amps": args.tile} if args.tile and fuse == "tile" else {}
    if args.block_dim:
        opts["block_dim"] = args.block_dim
    if fuse == "block":
        opts["tc_mode"] = args.tc_mode
    st.run(circ, fuse=fuse, **opts)
    st.synchronize()
    st.close()
    torch.cuda.synchronize()
    return 0


def run_ncu_block_case(args):
    """One 64-dimensional Haar block (the six highest wires) on 2^27 qubit
    amplitudes (1.07 GB complex64), applied twice in BF16x3: a case of the
    tile-ring kernel small enough for a full profiler capture (the second
    launch), larger than L2."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2410_17876_gb300 import binding as qb
    from paper_2410_17876_gb300 import inputs as gen

    st = qb.State((2,) * 27, prec=qb.QD_C64)
    st.set_fusion(1, "bf16x3")
    g = gen.Gate((21, 22, 23, 24, 25, 26), gen.haar(64, np.random.Generator(np.random.PCG64(1))))
    st.apply(g)
    st.apply(g)
    torch.cuda.synchronize()
    st.close()
    return 0


def run_ncu_batch_case(args):
    """The first 1024 circuits of the 8192-circuit workload, once through the
    device-side layer queue (a profiler capture of k_fused_layer)."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2410_17876_gb300 import binding as qb
    from paper_2410_17876_gb300 import inputs as gen

    circs = gen.config3_batch(n_circuits=1024)
    b = qb.qd_batch_create(qb.QD_C64)
    qb.qd_batch_run(b, circs, path=qb.QD_BATCH_LAYERS)
    qb.qd_batch_synchronize(b)
    qb.qd_batch_destroy(b)
    torch.cuda.synchronize()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--prec", choices=["c64", "c128"], default="c64",
                    help="precision of the profiler cases (the bench line itself is complex64; complex128 is "
                         "reported under benchmark_circuit)")
    ap.add_argument("--tc-mode", default="tf32x3", choices=["tf32x3", "bf16x3", "fp32"],
                    help="arithmetic of complex64 blocks of 17..64 dimensions when --fuse is not auto")
    ap.add_argument("--block-dim", type=int, default=0,
                    help="largest composed block with --fuse tile|block (0 = library default)")
    ap.add_argument("--ncu-workload", choices=["benchmark", "prefix"], default="benchmark",
                    help="profiler case: the 12-qubit + 8-qutrit benchmark circuit, or the 20-wire prefix of the "
                         "large workload (17,915,904 amplitudes, Haar gates)")
    ap.add_argument("--fuse", choices=["auto", "tile", "block", "off"], default="auto",
                    help="tile: consecutive gates share one shared-memory pass over the state; off: one pass per "
                         "gate; auto: the autotuner's choice of the two (and of tile size and block width)")
    ap.add_argument("--tile", type=int, default=0, help="amplitudes per fused tile (0 = library default)")
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the large-state and batched measurements")
    ap.add_argument("--ncu-case", action="store_true",
                    help="run only six dense single-wire gates (wires 0, 5, 10, 15, 19, 3) on the workload's "
                         "state, for a profiler capture of launches 4-6; prints nothing")
    ap.add_argument("--ncu-fused-case", action="store_true",
                    help="run only the --ncu-workload circuit once, fused (--fuse tile or block; auto means "
                         "tile), for a profiler capture of one fused launch; prints nothing")
    ap.add_argument("--ncu-block-case", action="store_true",
                    help="run only one 64-dimensional BF16x3 block twice on 2^27 amplitudes, for a profiler "
                         "capture of the tile-ring kernel; prints nothing")
    ap.add_argument("--ncu-batch-case", action="store_true",
                    help="run only 1024 circuits of the batched workload once through the layer queue, for a "
                         "profiler capture of the layer kernel; prints nothing")
    args = ap.parse_args(argv)
    if args.ncu_batch_case:
        return run_ncu_batch_case(args)
    if args.ncu_block_case:
        return run_ncu_block_case(args)
    if args.ncu_case:
        return run_ncu_case(args)
    if args.ncu_fused_case:
        return run_ncu_fused_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
