"""Pins of the sparse oracle (oracle/sparse.py): it equals the dense oracle
on random circuits of single-wire and controlled gates, and gives the GHZ
closed form at the sizes of the paper's sparse runs (62 qubits, 39 qutrits,
31 ququads, 27 ququints) and beyond 64-bit indices."""
import math

import numpy as np
import pytest

import oracle
from oracle import sparse
from paper_2410_17876_gb300 import inputs as gen


def random_single_wire_circuit(dims, depth, rng, p_dense=0.3):
    gates = []
    for _ in range(depth):
        t = int(rng.integers(0, len(dims)))
        d = dims[t]
        k = rng.random()
        if k < p_dense:
            U = gen.haar(d, rng)
        elif k < 0.6:
            U = gen.x_plus(d, int(rng.integers(1, d)))
        else:
            U = np.diag(np.exp(2j * np.pi * rng.random(d)))
        if rng.random() < 0.4:
            c = int(rng.integers(0, len(dims)))
            if c != t:
                gates.append(gen.Gate((t,), U, (c,), (int(rng.integers(0, dims[c])),)))
                continue
        gates.append(gen.Gate((t,), U))
    return gen.Circuit(tuple(dims), gates)


@pytest.mark.parametrize("seed", range(4))
def test_sparse_oracle_equals_dense_oracle(seed):
    rng = np.random.Generator(np.random.PCG64(900 + seed))
    dims = tuple(int(x) for x in rng.choice([2, 3, 4, 5], size=5))
    circ = random_single_wire_circuit(dims, 40, rng)
    dense = oracle.run_circuit(circ)
    sp = sparse.to_dense(dims, sparse.run_circuit(circ))
    assert np.max(np.abs(sp - dense)) < 1e-13


@pytest.mark.parametrize("d,n", [(2, 62), (3, 39), (4, 31), (5, 27), (2, 127), (3, 64)])
def test_sparse_oracle_ghz_closed_form(d, n):
    dims = (d,) * n
    st = sparse.run_circuit(gen.ghz_circuit(dims))
    b = sparse.strides(dims)
    expect = {k * sum(b[:n]): 1 / math.sqrt(d) for k in range(d)}
    assert set(st) == set(expect)
    for k, v in expect.items():
        assert abs(st[k] - v) < 1e-15


def test_sparse_oracle_drops_exact_zeros():
    dims = (2, 3)
    h = 1 / math.sqrt(2.0)
    H = np.array([[h, h], [h, -h]], dtype=np.complex128)  # exactly real: H H cancels exactly
    circ = gen.Circuit(dims, [gen.Gate((0,), H), gen.Gate((0,), H)])
    st = sparse.run_circuit(circ)
    assert set(st) == {0}
