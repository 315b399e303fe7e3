"""GPU parity of the tensor-core block path (tcgen05, complex64) and of the
whole-circuit block mode against the oracle: multi-wire gates of 17 to 64
dimensions (with controls, a ragged last chunk, odd strides), composed
blocks of random circuits, the 26.9M-amplitude benchmark circuit and the
20-wire prefix of the large workload."""
import numpy as np
import pytest

import __graft_entry__
import oracle
from tests.gpu_util import assert_close

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


def _run(qb, dims, gates, psi0, prec):
    st = qb.State(dims, prec=prec)
    st.set_amplitudes(psi0)
    for g in gates:
        st.apply(g)
    out = st.amplitudes()
    st.close()
    return out


def test_tc_single_block_small(qb, gen):
    """One 64-dimensional gate (three ququarts) on a 4 x 4 x 4 x 2 x 3 state."""
    rng = np.random.Generator(np.random.PCG64(1))
    dims = (4, 4, 4, 2, 3)
    psi0 = gen.random_state(int(np.prod(dims)), rng)
    g = gen.Gate((0, 1, 2), gen.haar(64, rng))
    got = _run(qb, dims, [g], psi0, qb.QD_C64)
    ref = oracle.apply_gate(dims, psi0, g)
    assert_close(got, ref, qb.QD_C64, "tc P=64")


@pytest.mark.parametrize("wires,extra", [((3, 0, 5), ()), ((1, 3, 4), ((2,), (1,))), ((0, 2, 6), ()),
                                         ((5, 6, 7), ((0,), (2,))), ((2, 3, 4, 7), ()), ((3, 6, 2, 4), ()),
                                         ((0, 1, 2), ((9,), (1,)))])
def test_tc_block_sizes_and_controls(qb, gen, wires, extra):
    rng = np.random.Generator(np.random.PCG64(sum(wires)))
    dims = (3, 3, 2, 4, 2, 3, 4, 2, 2, 3)
    P = int(np.prod([dims[w] for w in wires]))
    assert 17 <= P <= 64
    psi0 = gen.random_state(int(np.prod(dims)), rng)
    cw, cv = extra if extra else ((), ())
    g = gen.Gate(wires, gen.haar(P, rng), cw, cv)
    got = _run(qb, dims, [g, g], psi0, qb.QD_C64)
    ref = oracle.apply_gate(dims, oracle.apply_gate(dims, psi0, g), g)
    assert_close(got, ref, qb.QD_C64, f"tc wires={wires} P={P}")


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_block_mode_random_circuits(qb, gen, prec, seed):
    p = qb.QD_C64 if prec == "c64" else qb.QD_C128
    rng = np.random.Generator(np.random.PCG64(200 + seed))
    dims = tuple(int(x) for x in rng.choice([2, 3, 4], size=int(rng.integers(8, 12))))
    circ = gen.random_mixed_circuit(dims, 150, rng)
    psi0 = gen.random_state(circ.D, rng)
    st = qb.State(dims, prec=p)
    st.set_amplitudes(psi0)
    st.run(circ, fuse="block")
    got = st.amplitudes()
    st.close()
    assert_close(got, oracle.run_circuit(circ, psi0), p, f"block mode dims={dims}")


def test_block_mode_config2_prefix(qb, gen):
    pre = gen.prefix_circuit(gen.config2_circuit(), 20)
    ref = oracle.run_circuit(pre, nthreads=max(1, oracle.max_threads()))
    st = qb.State(pre.dims, prec=qb.QD_C64)
    st.run(pre, fuse="block")
    got = st.raw()
    st.close()
    assert_close(got, ref, qb.QD_C64, "config2 prefix, block mode")
