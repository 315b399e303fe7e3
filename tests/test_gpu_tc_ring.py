"""GPU parity of the BF16x3 tile-ring kernel (complex64 blocks of 9..64
dimensions without controls) against the oracle: tiles of up to 512
classes cut into chunks of 128 (the last one partial: 243, 216 and 144
classes), one to four chunks per tile, two to six ring slots, odd row lengths (8-byte copies instead
of bulk copies), a single tile holding the whole state, several tiles per
CTA with a ragged last round, blocks whose wires sit inside and above the
contiguous run, padded block dimensions, the launch counter that tells the
ring kernel from the register-staged one, and the bounded-wait timeout
path."""
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


def _apply(qb, dims, gates, psi0):
    st = qb.State(dims, prec=qb.QD_C64)
    st.set_fusion(1, "bf16x3")
    st.set_amplitudes(psi0)
    n0 = qb.qd_test_tc_ring_launches()
    for g in gates:
        st.apply(g)
    out = st.amplitudes()
    st.close()
    return out, qb.qd_test_tc_ring_launches() - n0


# (dims, block wires): run / row placement of the block's wires, class counts
CASES = [
    # the block above the run (128 classes, two slots of 64 KB)
    ((2,) * 7 + (2, 2, 2, 2, 2, 2) + (3, 2), (7, 8, 9, 10, 11, 12)),
    # odd row length: the lowest wires are qutrits (81 classes, 8-byte copies)
    ((3, 3, 3, 3, 3, 2, 2, 2, 2, 2, 2), (5, 6, 7, 8, 9)),
    # block wires interleaved with the run and above it (members inside and across rows)
    ((2, 3, 2, 4, 2, 3, 2, 2, 3, 2, 2), (0, 3, 6, 9)),
    # the block's wires listed out of order (member digits follow the gate's order)
    ((2, 2, 3, 2, 3, 2, 2, 3, 2, 2), (8, 1, 4, 0)),
    # P = 18 (padded to 24 rows of the operand), P = 54 (padded to 56)
    ((2, 2, 2, 3, 2, 3, 2, 2, 2, 2), (0, 3, 5)),
    ((2, 3, 3, 3, 2, 2, 2, 2, 2, 2), (0, 1, 2, 3)),
    # P = 27 (three qutrits), highest wires, 128 classes
    ((2, 2, 2, 2, 2, 2, 2, 3, 3, 3), (7, 8, 9)),
    # the whole state one tile (6 classes)
    ((4, 4, 4, 2, 3), (0, 1, 2)),
    # P = 48 on wires 0..2, the classes above the block
    ((4, 3, 4, 2, 3, 2, 2, 2, 3), (0, 1, 2)),
    # P = 9 and P = 16 (padded to 16 rows of the operand)
    ((2, 2, 3, 2, 2, 3, 2, 2, 2, 2, 2), (2, 5)),
    ((2, 3, 2, 2, 4, 2, 2, 2, 2, 2, 3, 2, 2), (4, 8, 7)),
    # several chunks of classes per tile (512 = 4 x 128, 16 tiles; 384 = 3 x 128 with qutrits among the class wires)
    ((2,) * 12 + (3, 4, 2, 2), (12, 13, 0)),
    ((2, 2, 2, 2, 2, 2, 2, 3, 2, 3, 2, 2, 2), (9, 12, 0, 1)),
]


@pytest.mark.parametrize("dims,wires", CASES)
def test_ring_block_matches_oracle(qb, gen, dims, wires):
    rng = np.random.Generator(np.random.PCG64(sum(dims) + 7 * len(wires)))
    P = int(np.prod([dims[w] for w in wires]))
    assert 9 <= P <= 64
    psi0 = gen.random_state(int(np.prod(dims)), rng)
    g = gen.Gate(wires, gen.haar(P, rng))
    got, ring = _apply(qb, dims, [g, g], psi0)
    ref = oracle.apply_gate(dims, oracle.apply_gate(dims, psi0, g), g)
    assert ring == 2, "both applications ran on the ring kernel"
    assert_close(got, ref, qb.QD_C64, f"ring dims={dims} wires={wires}")


def test_ring_many_tiles_per_cta(qb, gen):
    """2.65M amplitudes, a 64-dimensional block: 288 tiles of 144 classes
    (chunks of 128 and 16), several per CTA, a ragged last round over the SMs."""
    rng = np.random.Generator(np.random.PCG64(90))
    dims = (2, 3, 2, 2, 3, 2, 2, 2, 2, 3, 2, 2, 2, 2, 3, 2, 2, 2, 2)
    psi0 = gen.random_state(int(np.prod(dims)), rng)
    g = gen.Gate((2, 6, 10, 12, 13, 15), gen.haar(64, rng))
    got, ring = _apply(qb, dims, [g], psi0)
    assert ring == 1
    assert_close(got, oracle.apply_gate(dims, psi0, g), qb.QD_C64, "ring 2.65M amplitudes")


def test_controlled_blocks_take_the_register_staged_kernel(qb, gen):
    rng = np.random.Generator(np.random.PCG64(91))
    dims = (3, 3, 2, 4, 2, 3, 4, 2, 2, 3)
    psi0 = gen.random_state(int(np.prod(dims)), rng)
    g = gen.Gate((1, 3, 4), gen.haar(24, rng), (2,), (1,))
    got, ring = _apply(qb, dims, [g], psi0)
    assert ring == 0
    assert_close(got, oracle.apply_gate(dims, psi0, g), qb.QD_C64, "controlled block")


def test_ring_block_mode_circuit(qb, gen):
    """A random circuit in block mode (composed blocks of up to 64
    dimensions) with BF16x3: the tensor-core blocks run on the ring."""
    rng = np.random.Generator(np.random.PCG64(92))
    dims = (2, 3, 2, 2, 3, 2, 2, 3, 2, 2, 2, 3)
    c = gen.random_mixed_circuit(dims, 120, rng)
    st = qb.State(dims, prec=qb.QD_C64)
    n0 = qb.qd_test_tc_ring_launches()
    st.run(c, fuse="block", block_dim=64, tc_mode="bf16x3")
    got = st.amplitudes()
    ring = qb.qd_test_tc_ring_launches() - n0
    st.close()
    assert ring > 0
    assert_close(got, oracle.run_circuit(c), qb.QD_C64, "block mode bf16x3")


def test_ring_timeout_is_reported_and_the_state_recovers(qb, gen):
    """The ring kernel's bounded waits: with its loader copying nothing and a
    short poll limit, the converters' first waits run out; the kernel writes
    nothing, releases its tensor memory and returns, the next readout reports
    QD_ERR_TIMEOUT, and the same gate afterwards matches the oracle."""
    rng = np.random.Generator(np.random.PCG64(93))
    dims = (2, 2, 2, 2, 2, 3, 3, 2, 2, 3, 2, 2)
    psi0 = gen.random_state(int(np.prod(dims)), rng)
    g = gen.Gate((5, 6, 9), gen.haar(27, rng))
    st = qb.State(dims, prec=qb.QD_C64)
    st.set_fusion(1, "bf16x3")
    st.set_amplitudes(psi0)
    before = st.raw().copy()
    n0 = qb.qd_test_tc_ring_launches()
    try:
        qb.qd_test_set_tc_wait(1 << 12, stall_producers=True)
        st.apply(g)
        with pytest.raises(qb.QuditError) as ei:
            st.norm()
        assert ei.value.status == qb.QD_ERR_TIMEOUT, ei.value
    finally:
        qb.qd_test_set_tc_wait(0, stall_producers=False)
    assert qb.qd_test_tc_ring_launches() - n0 == 1
    assert np.array_equal(st.raw(), before)
    st.apply(g)
    got = st.amplitudes()
    assert abs(st.norm() - 1.0) < 1e-5
    st.close()
    assert_close(got, oracle.apply_gate(dims, before.astype(np.complex128), g), qb.QD_C64, "after a timeout")
