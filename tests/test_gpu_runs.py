"""Runs of single-wire gates applied in registers inside complex64 tile passes
(kRun, qubit blocks of three and four wires) and composed blocks of the other
shapes: gates with controls inside the block, diagonal and permutation gates
among them; results against the FP64 oracle."""
import numpy as np
import pytest

import __graft_entry__
import oracle
from tests.gpu_util import assert_close

pytestmark = pytest.mark.gpu

SHAPES = [(2, 2), (2, 3), (3, 2), (3, 3), (2, 2, 2), (2, 2, 3), (2, 3, 2), (3, 2, 2), (2, 2, 2, 2)]


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


def _run_circuit(gen, dims, nb, rng, rounds=2):
    """On the block wires 0..nb-1: a dense gate per wire, then controlled
    shifts along the chain and a phase gate, repeated; a gate on a wire
    outside the block between rounds."""
    gates = []
    for _ in range(rounds):
        for w in range(nb):
            gates.append(gen.Gate((w,), gen.haar(dims[w], rng)))
        for w in range(nb - 1):
            gates.append(gen.Gate((w + 1,), gen.x_plus(dims[w + 1], 1), (w,), (int(rng.integers(0, dims[w])),)))
        gates.append(gen.Gate((0,), np.diag(np.exp(2j * np.pi * rng.random(dims[0])))))
        gates.append(gen.Gate((0,), gen.x_plus(dims[0], 1), (nb - 1,), (1,)))
        w = int(rng.integers(nb, len(dims)))
        gates.append(gen.Gate((w,), gen.haar(dims[w], rng)))
    return gen.Circuit(dims, gates)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("seed", range(2))
def test_runs_match_oracle(qb, gen, shape, seed):
    rng = np.random.Generator(np.random.PCG64(900 + seed))
    dims = tuple(shape) + (2, 3, 2, 2, 3)
    circ = _run_circuit(gen, dims, len(shape), rng)
    psi0 = gen.random_state(circ.D, rng)
    for bd in (8, 16):
        st = qb.State(dims, prec=qb.QD_C64)
        st.set_amplitudes(psi0)
        st.run(circ, fuse="tile", block_dim=bd, max_tile_amps=1024)
        assert_close(st.amplitudes(), oracle.run_circuit(circ, psi0), qb.QD_C64, f"runs {shape} bd {bd}")
        st.close()


def test_runs_are_used_for_sparse_qubit_blocks(qb, gen):
    """Four qubits with one dense gate each and controlled shifts: a run is
    cheaper than the composed 16 x 16 block, so the complex64 plan counts each
    gate's own arithmetic (the complex128 plan, which has no runs, counts the
    composed product or single gates), and the result matches the oracle."""
    rng = np.random.Generator(np.random.PCG64(950))
    dims = (2, 2, 2, 2, 3, 2, 3)
    gates = [gen.Gate((w,), gen.haar(2, rng)) for w in range(4)]
    gates += [gen.Gate(((w + 1) % 4,), gen.x_plus(2, 1), (w,), (1,)) for w in range(4)]
    circ = gen.Circuit(dims, gates)
    f64 = qb.qd_plan_circuit(dims, qb.QD_C64, circ, mode=qb.QD_FUSE_TILE, max_tile_amps=1024, with_flops=True)[3]
    f128 = qb.qd_plan_circuit(dims, qb.QD_C128, circ, mode=qb.QD_FUSE_TILE, max_tile_amps=1024, with_flops=True)[3]
    assert sum(f64) != sum(f128)
    psi0 = gen.random_state(circ.D, rng)
    st = qb.State(dims, prec=qb.QD_C64)
    st.set_amplitudes(psi0)
    st.run(circ, fuse="tile", max_tile_amps=1024)
    assert_close(st.amplitudes(), oracle.run_circuit(circ, psi0), qb.QD_C64, "sparse qubit run")
    st.close()
