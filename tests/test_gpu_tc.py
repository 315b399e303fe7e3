"""GPU parity of the tensor-core block path (tcgen05, complex64) and of the
whole-circuit block mode against the oracle: multi-wire gates of 17 to 64
dimensions (with controls, a ragged last chunk, odd strides) in each block
arithmetic (TF32x3 and BF16x3 tensor-core products, FP32 CUDA cores),
composed blocks of random circuits, deferred fusion of single-gate calls,
and the 20-wire prefix of the large workload with the error of each
arithmetic against the FP64 oracle."""
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


TC_MODES = ["tf32x3", "bf16x3", "fp32"]


def _run(qb, dims, gates, psi0, prec, tc_mode="tf32x3"):
    st = qb.State(dims, prec=prec)
    st.set_fusion(1, tc_mode)  # no deferral; tc_mode picks the arithmetic of gates of 17..64 dimensions
    st.set_amplitudes(psi0)
    for g in gates:
        st.apply(g)
    out = st.amplitudes()
    st.close()
    return out


@pytest.mark.parametrize("tc_mode", TC_MODES)
def test_tc_single_block_small(qb, gen, tc_mode):
    """One 64-dimensional gate (three ququarts) on a 4 x 4 x 4 x 2 x 3 state."""
    rng = np.random.Generator(np.random.PCG64(1))
    dims = (4, 4, 4, 2, 3)
    psi0 = gen.random_state(int(np.prod(dims)), rng)
    g = gen.Gate((0, 1, 2), gen.haar(64, rng))
    got = _run(qb, dims, [g], psi0, qb.QD_C64, tc_mode)
    ref = oracle.apply_gate(dims, psi0, g)
    assert_close(got, ref, qb.QD_C64, f"{tc_mode} P=64")


def test_tc_modes_differ_by_their_rounding(qb, gen):
    """The three arithmetics are separate paths: their results are not
    bit-identical, and each error against the oracle is within its own
    bound (TF32x3 ~2^-21, BF16x3 ~2^-16 relative per block)."""
    rng = np.random.Generator(np.random.PCG64(5))
    dims = (4, 4, 4, 2, 3, 2)
    psi0 = gen.random_state(int(np.prod(dims)), rng)
    g = gen.Gate((1, 2, 0), gen.haar(64, rng))
    ref = oracle.apply_gate(dims, psi0, g)
    outs = {m: _run(qb, dims, [g], psi0, qb.QD_C64, m) for m in TC_MODES}
    rel = {m: float(np.linalg.norm(outs[m] - ref) / np.linalg.norm(ref)) for m in TC_MODES}
    assert rel["tf32x3"] < 2e-6 and rel["fp32"] < 2e-6, rel
    assert rel["bf16x3"] < 1e-4, rel
    assert not np.array_equal(outs["tf32x3"], outs["bf16x3"])
    assert not np.array_equal(outs["tf32x3"], outs["fp32"])


@pytest.mark.parametrize("tc_mode", TC_MODES)
def test_tc_no_norm_drift(qb, gen, tc_mode):
    """40 applications of a 64-dimensional unitary: the state's norm stays 1
    (the tensor cores' FP32 accumulation is biased toward zero; unitary
    blocks restore each class's norm) and the amplitudes match the oracle."""
    rng = np.random.Generator(np.random.PCG64(7))
    dims = (4, 4, 4, 2, 3, 2, 2, 2)
    psi0 = gen.random_state(int(np.prod(dims)), rng)
    g = gen.Gate((0, 1, 2), gen.haar(64, rng))
    st = qb.State(dims, prec=qb.QD_C64)
    st.set_fusion(1, tc_mode)
    st.set_amplitudes(psi0)
    ref = psi0
    for _ in range(40):
        st.apply(g)
        ref = oracle.apply_gate(dims, ref, g)
    assert abs(st.norm() - 1.0) < 2e-6
    assert_close(st.amplitudes(), ref, qb.QD_C64, f"{tc_mode} x40")
    st.close()


@pytest.mark.parametrize("tc_mode", TC_MODES)
def test_tc_non_unitary_block_is_not_rescaled(qb, gen, tc_mode):
    """A non-unitary 48-dimensional matrix (0.7 x a Haar unitary, plus a
    rank-one term) is applied as given: the result follows the matrix, not
    a renormalised version of it."""
    rng = np.random.Generator(np.random.PCG64(8))
    dims = (4, 3, 4, 2, 3, 2)
    psi0 = gen.random_state(int(np.prod(dims)), rng)
    M = 0.7 * gen.haar(48, rng)
    M[:, 0] += 0.2
    g = gen.Gate((0, 1, 2), M)
    got = _run(qb, dims, [g], psi0, qb.QD_C64, tc_mode)
    ref = oracle.apply_gate(dims, psi0, g)
    assert abs(np.linalg.norm(ref) - 1.0) > 0.1
    assert_close(got, ref, qb.QD_C64, f"{tc_mode} non-unitary")


@pytest.mark.parametrize("tc_mode", TC_MODES)
@pytest.mark.parametrize("wires,extra", [((3, 0, 5), ()), ((1, 3, 4), ((2,), (1,))), ((0, 2, 6), ()),
                                         ((5, 6, 7), ((0,), (2,))), ((2, 3, 4, 7), ()), ((3, 6, 2, 4), ()),
                                         ((0, 1, 2), ((9,), (1,)))])
def test_tc_block_sizes_and_controls(qb, gen, wires, extra, tc_mode):
    rng = np.random.Generator(np.random.PCG64(sum(wires)))
    dims = (3, 3, 2, 4, 2, 3, 4, 2, 2, 3)
    P = int(np.prod([dims[w] for w in wires]))
    assert 17 <= P <= 64
    psi0 = gen.random_state(int(np.prod(dims)), rng)
    cw, cv = extra if extra else ((), ())
    g = gen.Gate(wires, gen.haar(P, rng), cw, cv)
    got = _run(qb, dims, [g, g], psi0, qb.QD_C64, tc_mode)
    ref = oracle.apply_gate(dims, oracle.apply_gate(dims, psi0, g), g)
    assert_close(got, ref, qb.QD_C64, f"{tc_mode} wires={wires} P={P}")


@pytest.mark.parametrize("prec,tc_mode", [("c64", "tf32x3"), ("c64", "bf16x3"), ("c64", "fp32"),
                                          ("c128", "tf32x3")])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_block_mode_random_circuits(qb, gen, prec, tc_mode, seed):
    p = qb.QD_C64 if prec == "c64" else qb.QD_C128
    rng = np.random.Generator(np.random.PCG64(200 + seed))
    dims = tuple(int(x) for x in rng.choice([2, 3, 4], size=int(rng.integers(8, 12))))
    circ = gen.random_mixed_circuit(dims, 150, rng)
    psi0 = gen.random_state(circ.D, rng)
    st = qb.State(dims, prec=p)
    st.set_amplitudes(psi0)
    st.run(circ, fuse="block", tc_mode=tc_mode)
    nrm = st.norm()
    got = st.amplitudes()
    st.close()
    assert_close(got, oracle.run_circuit(circ, psi0), p, f"block mode {tc_mode} dims={dims}")
    # no systematic drift of the norm (unbiased rounding of the split operands)
    assert abs(nrm - 1.0) < (1e-12 if p == qb.QD_C128 else 1e-5), nrm


@pytest.mark.parametrize("tc_mode", TC_MODES)
def test_deferred_fusion(qb, gen, tc_mode):
    """qd_set_fusion queues single-gate calls; readouts flush the queue, and
    set_amplitudes discards it."""
    rng = np.random.Generator(np.random.PCG64(31))
    dims = (2, 3, 4, 2, 3, 2, 2, 3, 4)
    circ = gen.random_mixed_circuit(dims, 120, rng)
    psi0 = gen.random_state(circ.D, rng)
    st = qb.State(dims, prec=qb.QD_C64)
    st.set_fusion(64, tc_mode)
    st.set_amplitudes(psi0)
    launches = qb.qd_launch_count()
    st.run_gate_by_gate(circ)
    assert qb.qd_launch_count() == launches  # queued, nothing launched
    assert abs(st.norm() - 1.0) < 1e-5       # the readout flushes
    assert qb.qd_launch_count() > launches
    got = st.amplitudes()
    assert_close(got, oracle.run_circuit(circ, psi0), qb.QD_C64, f"deferred {tc_mode}")
    # queued gates are dropped by set_amplitudes (the state is overwritten)
    st.run_gate_by_gate(circ)
    st.set_amplitudes(psi0)
    assert np.max(np.abs(st.amplitudes() - psi0)) < 1e-7
    # explicit flush, then back to one launch per call
    half = gen.Circuit(dims, circ.gates[:60])
    st.run_gate_by_gate(half)
    st.flush()
    st.set_fusion(1, tc_mode)
    st.run_gate_by_gate(gen.Circuit(dims, circ.gates[60:]))
    assert_close(st.amplitudes(), oracle.run_circuit(circ, psi0), qb.QD_C64, f"deferred+flush {tc_mode}")
    st.close()


@pytest.fixture(scope="module")
def config2_prefix(gen):
    pre = gen.prefix_circuit(gen.config2_circuit(), 20)
    return pre, oracle.run_circuit(pre, nthreads=max(1, oracle.max_threads()))


@pytest.mark.parametrize("tc_mode", TC_MODES)
def test_block_mode_config2_prefix(qb, config2_prefix, tc_mode):
    pre, ref = config2_prefix
    st = qb.State(pre.dims, prec=qb.QD_C64)
    st.run(pre, fuse="block", tc_mode=tc_mode)
    got = st.raw()
    st.close()
    assert_close(got, ref, qb.QD_C64, f"config2 prefix, block mode {tc_mode}")


def test_tc_wait_timeout_is_reported_and_the_state_recovers(qb, gen):
    """The timeout path of the tensor-core block kernel, without a GPU fault:
    with its producers kept from publishing and a short poll limit, every
    CTA's first bounded wait runs out; the kernel writes nothing, releases its
    tensor memory and returns, and the next readout reports QD_ERR_TIMEOUT.
    The state is unchanged, and the same gate applied afterwards with the
    default limits matches the oracle."""
    rng = np.random.Generator(np.random.PCG64(41))
    dims = (2, 2, 2, 2, 2, 3, 3, 2, 2, 3, 2, 2)  # 5 qubit wires form a 32-dimensional gate
    psi0 = gen.random_state(int(np.prod(dims)), rng)
    g = gen.Gate((0, 1, 2, 3, 4), gen.haar(32, rng))
    st = qb.State(dims, prec=qb.QD_C64)
    st.set_fusion(1, "tf32x3")
    st.set_amplitudes(psi0)
    before = st.raw().copy()
    try:
        qb.qd_test_set_tc_wait(1 << 12, stall_producers=True)
        st.apply(g)
        with pytest.raises(qb.QuditError) as ei:
            st.norm()
        assert ei.value.status == qb.QD_ERR_TIMEOUT, ei.value
    finally:
        qb.qd_test_set_tc_wait(0, stall_producers=False)
    assert np.array_equal(st.raw(), before)  # the stalled pass wrote nothing
    st.apply(g)
    got = st.amplitudes()
    assert abs(st.norm() - 1.0) < 1e-5
    st.close()
    assert_close(got, oracle.apply_gate(dims, before.astype(np.complex128), g), qb.QD_C64, "after a timeout")
