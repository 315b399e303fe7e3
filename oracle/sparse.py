"""Sparse FP64 oracle: a state as a dict {basis index: amplitude}.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests and the
benchmark's CPU leg may use it; the product library never does.  It shares
no code with the CUDA path.

It follows the paper's remark that a unitary is applied by inspecting the
indices of the non-zero amplitudes only (end of section "Example Circuit";
the sparse columns of the experiments): for every stored index j whose
control digits floor(j / b_c) mod d_c all equal their values, with target
digit x = floor(j / b_t) mod d_t, the amplitude a_j is sent to the d_t
indices j + (r - x) b_t with weight U[r, x]; contributions to the same index
are summed (in the order the stored indices are visited, which is ascending);
indices whose controls are not met keep their amplitude.  Exact zeros are
dropped.  Indices are Python integers, so there is no limit on D.
"""
from __future__ import annotations

from typing import Dict, Sequence

import numpy as np


def strides(dims: Sequence[int]):
    b = [1]
    for d in dims:
        b.append(b[-1] * int(d))
    return b  # b[w] = d_0 ... d_{w-1}; b[n] = D


def zero_state() -> Dict[int, complex]:
    return {0: 1 + 0j}


def apply_gate(dims: Sequence[int], state: Dict[int, complex], gate) -> Dict[int, complex]:
    """One single-wire gate (optionally controlled) on a sparse state."""
    if len(gate.wires) != 1:
        raise ValueError("the sparse oracle takes single-wire gates")
    b = strides(dims)
    t = int(gate.wires[0])
    d = int(dims[t])
    U = np.asarray(gate.U, dtype=np.complex128)
    ctrl = [(int(w), int(v)) for w, v in zip(gate.controls, gate.values)]
    out: Dict[int, complex] = {}
    for j in sorted(state):
        a = state[j]
        if any((j // b[w]) % int(dims[w]) != v for w, v in ctrl):
            out[j] = out.get(j, 0j) + a
            continue
        x = (j // b[t]) % d
        base = j - x * b[t]
        for r in range(d):
            u = U[r, x]
            if u != 0:
                k = base + r * b[t]
                out[k] = out.get(k, 0j) + complex(u) * a
    return {k: v for k, v in out.items() if v != 0}


def run_circuit(circ, state=None) -> Dict[int, complex]:
    s = zero_state() if state is None else dict(state)
    for g in circ.gates:
        s = apply_gate(circ.dims, s, g)
    return s


def to_dense(dims: Sequence[int], state: Dict[int, complex]) -> np.ndarray:
    D = int(np.prod(np.asarray(dims, dtype=np.int64)))
    out = np.zeros(D, dtype=np.complex128)
    for k, v in state.items():
        out[k] = v
    return out
