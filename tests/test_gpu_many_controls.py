"""Gates with many controls: the digit-insertion enumeration of
qd_apply_controlled against the paper's scanning formulation
(qd_apply_controlled_scan, every target class visited and its control digits
tested).  Both give the same state bit for bit, and both match the oracle."""
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


DIMS = (2, 3, 2, 2, 3, 2, 5, 2, 3, 2, 2, 4, 2)


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("n_ctrl", [1, 2, 3, 5, 8, 12])
def test_scan_equals_enumeration(qb, gen, prec, n_ctrl):
    p = qb.QD_C64 if prec == "c64" else qb.QD_C128
    rng = np.random.Generator(np.random.PCG64(500 + n_ctrl))
    D = int(np.prod(DIMS))
    psi0 = gen.random_state(D, rng)
    gates = []
    for _ in range(6):
        t = int(rng.integers(0, len(DIMS)))
        others = [w for w in range(len(DIMS)) if w != t]
        cw = [int(w) for w in rng.permutation(others)[:n_ctrl]]
        cv = [int(rng.integers(0, DIMS[w])) for w in cw]
        U = gen.haar(DIMS[t], rng) if rng.random() < 0.5 else gen.x_plus(DIMS[t], 1)
        gates.append(gen.Gate((t,), U, tuple(cw), tuple(cv)))
    a = qb.State(DIMS, prec=p)
    b = qb.State(DIMS, prec=p)
    a.set_amplitudes(psi0)
    b.set_amplitudes(psi0)
    for g in gates:
        qb.qd_apply_controlled(a.handle, g.wires[0], g.U, g.controls, g.values)
        qb.qd_apply_controlled_scan(b.handle, g.wires[0], g.U, g.controls, g.values)
    ra, rb = a.raw(), b.raw()
    assert np.array_equal(ra, rb)
    ref = psi0
    for g in gates:
        ref = oracle.apply_gate(DIMS, ref, g)
    assert_close(a.amplitudes(), ref, p, f"{n_ctrl} controls")
    a.close()
    b.close()


def test_scan_then_inverse_by_enumeration(qb, gen):
    rng = np.random.Generator(np.random.PCG64(9))
    D = int(np.prod(DIMS))
    psi0 = gen.random_state(D, rng)
    st = qb.State(DIMS, prec=qb.QD_C128)
    st.set_amplitudes(psi0)
    before = st.raw()
    # a gate and its inverse on the same controls, one through each formulation
    qb.qd_apply_controlled_scan(st.handle, 0, gen.fourier(2), (1, 6), (2, 4))
    qb.qd_apply_controlled(st.handle, 0, np.conj(gen.fourier(2)).T, (1, 6), (2, 4))
    after = st.raw()
    assert np.max(np.abs(after - before)) < 1e-15
    st.close()


def test_scan_rejects_wide_target(qb):
    st = qb.State((2, 16, 2), prec=qb.QD_C64)
    with pytest.raises(qb.QuditError) as ei:
        qb.qd_apply_controlled_scan(st.handle, 1, np.eye(16, dtype=complex), (0,), (1,))
    assert ei.value.status == qb.QD_ERR_UNSUPPORTED
    st.close()
