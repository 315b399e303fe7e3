"""GPU sparse states (qd_sparse_*) against the sparse oracle, the dense
oracle and the GHZ closed form: random circuits of single-wire and
controlled gates, the paper's GHZ sizes (62 qubits, 39 qutrits, 31 ququads,
27 ququints), beyond 64-bit indices (127 qubits, 64 qutrits, 42 ququints),
exact cancellation, and the capacity limit."""
import math

import numpy as np
import pytest

import __graft_entry__
import oracle
from oracle import sparse
from tests.test_oracle_sparse import random_single_wire_circuit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qb():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    __graft_entry__.build()
    from paper_2410_17876_gb300 import binding

    return binding


@pytest.fixture(scope="module")
def gen():
    from paper_2410_17876_gb300 import inputs

    return inputs


def _run(qb, circ):
    s = qb.qd_sparse_create(circ.dims)
    qb.qd_sparse_run(s, circ)
    out = qb.qd_sparse_get(s)
    qb.qd_sparse_destroy(s)
    return out


@pytest.mark.parametrize("seed", range(6))
def test_random_circuits_match_oracles(qb, gen, seed):
    rng = np.random.Generator(np.random.PCG64(950 + seed))
    dims = tuple(int(x) for x in rng.choice([2, 3, 4, 5, 8], size=4))
    while np.prod(dims) > 512:
        dims = dims[:-1]
    circ = random_single_wire_circuit(dims, 60, rng)
    got = _run(qb, circ)
    ref = sparse.run_circuit(circ)
    dense = oracle.run_circuit(circ)
    assert len(got) <= qb.QD_SPARSE_MAX_NNZ
    assert set(got) <= set(range(int(np.prod(dims))))
    g = sparse.to_dense(dims, got)
    assert np.max(np.abs(g - dense)) < 1e-12
    assert np.max(np.abs(g - sparse.to_dense(dims, ref))) < 1e-12


def test_sparse_circuit_on_a_wide_basis(qb, gen):
    """30 wires of mixed dimension (D = 2^15 3^10 4^5 > 2^40), a sparse-friendly
    circuit (permutations, phases, a few dense gates) against the sparse oracle."""
    rng = np.random.Generator(np.random.PCG64(961))
    dims = tuple([2] * 15 + [3] * 10 + [4] * 5)
    dims = tuple(int(x) for x in rng.permutation(dims))
    circ = random_single_wire_circuit(dims, 120, rng, p_dense=0.05)
    got = _run(qb, circ)
    ref = sparse.run_circuit(circ)
    assert set(got) == set(ref)
    assert max(abs(got[k] - ref[k]) for k in ref) < 1e-12


@pytest.mark.parametrize("d,n", [(2, 62), (3, 39), (4, 31), (5, 27), (2, 127), (3, 64), (5, 42)])
def test_ghz_closed_form(qb, gen, d, n):
    dims = (d,) * n
    got = _run(qb, gen.ghz_circuit(dims))
    b = sparse.strides(dims)
    expect = {k * sum(b[:n]): 1 / math.sqrt(d) for k in range(d)}
    assert set(got) == set(expect)
    for k, v in expect.items():
        assert abs(got[k] - v) < 1e-15


def test_mixed_radix_ghz(qb, gen):
    dims = (3, 4, 5, 3, 8, 4, 3, 5)
    got = _run(qb, gen.ghz_circuit(dims, root=0))
    b = sparse.strides(dims)
    expect = {k * sum(b[:len(dims)]): 1 / math.sqrt(3) for k in range(3)}
    assert set(got) == set(expect)


def test_exact_cancellation(qb, gen):
    h = 1 / math.sqrt(2.0)
    H = np.array([[h, h], [h, -h]], dtype=np.complex128)
    circ = gen.Circuit((2, 3, 2), [gen.Gate((0,), H), gen.Gate((2,), H), gen.Gate((0,), H)])
    got = _run(qb, circ)
    assert set(got) == {0, 6}


def test_capacity_limit_leaves_the_state(qb, gen):
    dims = (2,) * 12
    H = gen.fourier(2)
    s = qb.qd_sparse_create(dims)
    qb.qd_sparse_run(s, gen.Circuit(dims, [gen.Gate((w,), H) for w in range(8)]))  # 256 entries
    before = qb.qd_sparse_get(s)
    with pytest.raises(qb.QuditError) as ei:
        qb.qd_sparse_run(s, gen.Circuit(dims, [gen.Gate((w,), H) for w in range(8, 10)]))  # 1024
    assert ei.value.status == qb.QD_ERR_UNSUPPORTED
    assert qb.qd_sparse_get(s) == before
    qb.qd_sparse_destroy(s)


def test_rejects_multi_wire_and_wide_dims(qb, gen):
    with pytest.raises(qb.QuditError):
        qb.qd_sparse_create((2, 16))
    with pytest.raises(qb.QuditError):
        qb.qd_sparse_create((2,) * 129)
    s = qb.qd_sparse_create((2, 2))
    with pytest.raises(qb.QuditError) as ei:
        qb.qd_sparse_run(s, gen.Circuit((2, 2), [gen.Gate((0, 1), np.eye(4, dtype=complex))]))
    assert ei.value.status == qb.QD_ERR_UNSUPPORTED
    qb.qd_sparse_destroy(s)


def test_grid_tier_matches_oracles(qb, gen):
    """Supports beyond the one-CTA buffers (qd_sparse_reserve): about 83K
    non-zero amplitudes on 16 wires, dense, controlled and permutation gates,
    against the sparse oracle and the dense oracle."""
    rng = np.random.Generator(np.random.PCG64(971))
    dims = (2, 3, 2, 2, 3, 2, 2, 2, 3, 2, 2, 2, 2, 3, 2, 2)
    gates = [gen.Gate((w,), gen.fourier(dims[w])) for w in range(0, 12)]
    gates += random_single_wire_circuit(dims, 40, rng).gates
    circ = gen.Circuit(dims, gates)
    s = qb.qd_sparse_create(dims)
    qb.qd_sparse_reserve(s, 1 << 18)
    qb.qd_sparse_run(s, circ)
    got = qb.qd_sparse_get(s)
    qb.qd_sparse_destroy(s)
    assert len(got) > qb.QD_SPARSE_MAX_NNZ
    ref = sparse.run_circuit(circ)
    assert set(got) == set(ref)
    assert max(abs(got[k] - ref[k]) for k in ref) < 1e-12
    dense = oracle.run_circuit(circ)
    assert np.max(np.abs(sparse.to_dense(dims, got) - dense)) < 1e-12


def test_grid_tier_round_trip_and_capacity(qb, gen):
    """The support grows past the one-CTA buffers and shrinks back (the state
    returns to the one-CTA path); an overflow of the reserved capacity leaves
    the state as before the call; a larger reservation keeps the state."""
    dims = (2,) * 14
    h = 1 / math.sqrt(2.0)
    H = np.array([[h, h], [h, -h]], dtype=np.complex128)  # exactly real: undoing it cancels exactly
    s = qb.qd_sparse_create(dims)
    qb.qd_sparse_reserve(s, 2048)
    qb.qd_sparse_run(s, gen.Circuit(dims, [gen.Gate((w,), H) for w in range(10)]))  # 1024 entries
    assert qb.qd_sparse_nnz(s) == 1024
    before = qb.qd_sparse_get(s)
    with pytest.raises(qb.QuditError) as ei:
        qb.qd_sparse_run(s, gen.Circuit(dims, [gen.Gate((w,), H) for w in range(10, 12)]))  # 4096 > 2048
    assert ei.value.status == qb.QD_ERR_UNSUPPORTED
    assert qb.qd_sparse_get(s) == before
    qb.qd_sparse_reserve(s, 8192)
    assert qb.qd_sparse_get(s) == before
    qb.qd_sparse_run(s, gen.Circuit(dims, [gen.Gate((w,), H) for w in range(10, 12)]))
    assert qb.qd_sparse_nnz(s) == 4096
    # undo all Hadamards: back to |0...0>, then a GHZ on the one-CTA path
    qb.qd_sparse_run(s, gen.Circuit(dims, [gen.Gate((w,), H) for w in range(12)]))
    got = qb.qd_sparse_get(s)
    assert set(got) == {0} and abs(got[0] - 1.0) < 1e-12
    qb.qd_sparse_run(s, gen.ghz_circuit(dims))
    got = qb.qd_sparse_get(s)
    assert set(got) == {0, 2 ** 14 - 1}
    with pytest.raises(qb.QuditError):
        qb.qd_sparse_reserve(s, 100)
    qb.qd_sparse_destroy(s)
