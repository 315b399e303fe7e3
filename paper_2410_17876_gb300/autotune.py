"""Autotuner for the fused path and the batch executor.

Picks the fused tile size (amplitudes per shared-memory tile) and the block
width (largest composed block) for a workload by timing candidates on the
GPU with CUDA events on the launching stream, and caches the choice in a
JSON file keyed by GPU name, precision and workload shape.  Given a cache
entry the choice is deterministic.  Timing runs go through the same C-ABI
calls as production runs; the tuner itself makes no numerical decision.

Cache file: ``$QD_TUNE_CACHE``, else ``~/.cache/qudit_gb300/autotune.json``.
"""
from __future__ import annotations

import json
import math
import os
import time
from typing import Callable, Dict, Iterable, Optional, Sequence, Tuple

import numpy as np

# (mode, max_tile_amps, block_dim, tc_mode): mode 0 = one kernel pass per
# gate, 1 = shared-memory tile passes, 2 = whole-state composed blocks;
# tc_mode = the arithmetic of complex64 blocks of 17..64 dimensions
# (0 TF32x3, 1 BF16x3).  Whole-state block candidates come first, so that a
# spent time budget cuts tile candidates, not them.
FUSION_CANDIDATES = {
    0: [(0, 0, 0, 0)] + [(2, 0, b, tc) for tc in (1, 0) for b in (64, 32)]
       + [(1, t, b, 0) for t in (2048, 4096, 8192, 16384) for b in (1, 4, 8, 16)]
       + [(1, t, b, 0) for t in (4096, 8192) for b in (24, 32)],  # blocks of 17..32 dims on tensor cores in tiles
    1: [(0, 0, 0, 0)] + [(1, t, b, 0) for t in (1024, 2048, 4096, 8192) for b in (1, 4, 8, 16)]
       + [(2, 0, b, 0) for b in (4, 8)],
}
TC_NAMES = {0: "tf32x3", 1: "bf16x3"}
MODE_NAMES = {0: "off", 1: "tile", 2: "block"}


def cache_path() -> str:
    p = os.environ.get("QD_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "qudit_gb300", "autotune.json")


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d: dict) -> None:
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def gpu_name() -> str:
    import torch

    return torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"


def shape_key(kind: str, prec: int, dims: Sequence[int], n_gates: int) -> str:
    """Workload signature: wires, log2 of the amplitude count, largest dimension, gate count bucket."""
    D = int(np.prod(np.asarray(dims, dtype=np.int64)))
    return (f"{gpu_name()}|{kind}|prec{prec}|n{len(dims)}|log2D{int(round(math.log2(max(D, 1))))}|"
            f"dmax{max(dims)}|g{int(round(math.log2(max(n_gates, 1))))}")


def time_candidates(run: Callable[[tuple], None], candidates: Iterable[tuple],
                    stream, reps: int = 3, budget_s: float = 30.0) -> Dict[tuple, float]:
    """Seconds per run of each candidate (one warm-up run, then ``reps`` timed
    with CUDA events on ``stream``); stops early when the budget is spent."""
    import torch

    out = {}
    t_start = time.perf_counter()
    for cand in candidates:
        if time.perf_counter() - t_start > budget_s:
            break
        run(cand)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run(cand)
        e1.record(stream)
        torch.cuda.synchronize()
        out[cand] = e0.elapsed_time(e1) / 1e3 / reps
    return out


def tune_circuit(state, circuit, retune: bool = False, reps: int = 3, budget_s: float = 30.0) -> dict:
    """Best fusion settings for ``circuit`` on ``state`` (a ``binding.State`` of
    the circuit's dims).  Returns {"mode" ("off" / "tile" / "block"),
    "max_tile_amps", "block_dim", "tc_mode" ("tf32x3" / "bf16x3"), "seconds",
    "table"}; the state is left in an unspecified state."""
    key = shape_key("circuit2", state.prec, circuit.dims, len(circuit.gates))
    cache = _load()
    if not retune and key in cache:
        return cache[key]

    def run(c):
        state.reset()
        if c[0] == 0:
            state.run(circuit, fuse=False)
        else:
            state.run(circuit, fuse=MODE_NAMES[c[0]], max_tile_amps=c[1], block_dim=c[2], tc_mode=TC_NAMES[c[3]])

    table = time_candidates(run, FUSION_CANDIDATES[state.prec], state.stream, reps=reps, budget_s=budget_s)
    best = min(table, key=table.get)
    entry = {"mode": MODE_NAMES[best[0]], "max_tile_amps": best[1], "block_dim": best[2],
             "tc_mode": TC_NAMES[best[3]], "seconds": table[best],
             "table": {f"{MODE_NAMES[m]}/{t}/{b}/{TC_NAMES[tc]}": v for (m, t, b, tc), v in table.items()}}
    cache[key] = entry
    _save(cache)
    return entry


def tune_batch(circuits, prec: int, stream, retune: bool = False, sample: int = 512,
               small_caps: Sequence[int] = (2048, 4096, 8192), block_dims: Sequence[int] = (4, 8, 16),
               paths: Sequence[int] = (0, 1), reps: int = 2, budget_s: float = 30.0) -> dict:
    """Best one-CTA threshold, block width and path (0: device-side layer
    queue, 1: one program per circuit on auxiliary streams) for a batch of
    circuits, timed on a seeded sample of the batch (graph relaunches)."""
    from . import binding as qb

    key = f"{gpu_name()}|batch2|prec{prec}|n{len(circuits)}"
    cache = _load()
    if not retune and key in cache:
        return cache[key]
    rng = np.random.Generator(np.random.PCG64(0))
    idx = rng.permutation(len(circuits))[:min(sample, len(circuits))]
    subset = [circuits[int(i)] for i in sorted(idx)]
    b = qb.qd_batch_create(prec, stream.cuda_stream)
    cands = [(s, bd, p) for p in paths for s in small_caps for bd in block_dims]
    if prec == qb.QD_C128:
        cands = [c for c in cands if c[0] <= 4096]
    state = {"c": None}

    def run(c):
        if state["c"] != c:
            qb.qd_batch_run(b, subset, small_max_amps=c[0], block_dim=c[1], use_graph=True, path=c[2])
            state["c"] = c
        else:
            qb.qd_batch_relaunch(b)

    table = time_candidates(run, cands, stream, reps=reps, budget_s=budget_s)
    qb.qd_batch_destroy(b)
    best = min(table, key=table.get)
    entry = {"small_max_amps": best[0], "block_dim": best[1], "path": best[2], "seconds_sample": table[best],
             "table": {f"{s}/{bd}/{p}": v for (s, bd, p), v in table.items()}}
    cache[key] = entry
    _save(cache)
    return entry
