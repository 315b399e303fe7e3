"""GPU parity at the workload sizes: full circuits against the oracle where
the oracle finishes in about a minute, properties that hold at any size
where it cannot (the 1.72e9-amplitude state)."""
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


@pytest.fixture(scope="module")
def config1_ref(gen):
    circ = gen.config1_circuit()
    return circ, oracle.run_circuit(circ, nthreads=max(1, oracle.max_threads()))


@pytest.mark.parametrize("fuse", [False, True])
@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_config1_full_depth_500(qb, config1_ref, prec, fuse):
    """12 qubits + 8 qutrits (26,873,856 amplitudes), 500 gates, gate by gate and fused."""
    circ, ref = config1_ref
    p = qb.QD_C128 if prec == "c128" else qb.QD_C64
    st = qb.State(circ.dims, prec=p)
    st.run(circ, fuse=fuse)
    got = st.raw()
    nrm = st.norm()
    st.close()
    assert_close(got, ref, p, f"config1 {prec}")
    assert abs(nrm - 1.0) < (1e-12 if p == qb.QD_C128 else 1e-5)


@pytest.mark.parametrize("fuse", [False, True])
def test_config2_prefix_against_oracle(qb, gen, fuse):
    """The lowest 20 wires of the 18-qubit + 8-qutrit workload with the gates that stay inside them."""
    full = gen.config2_circuit()
    pre = gen.prefix_circuit(full, 20)
    ref = oracle.run_circuit(pre, nthreads=max(1, oracle.max_threads()))
    st = qb.State(pre.dims, prec=qb.QD_C64)
    st.run(pre, fuse=fuse)
    got = st.raw()
    st.close()
    assert_close(got, ref, qb.QD_C64, "config2 prefix")


@pytest.mark.parametrize("fuse", [False, True])
def test_config2_full_size_inverse_returns_to_zero(qb, gen, fuse):
    """1.72e9 amplitudes, complex64: the circuit followed by its inverse gives
    back |0...0> (|psi_0|^2 = 1 and norm 1 pin every other amplitude to ~0)."""
    import torch

    circ = gen.config2_circuit()
    inv = gen.Circuit(circ.dims, [gen.Gate(g.wires, g.U.conj().T, g.controls, g.values)
                                  for g in reversed(circ.gates)])
    st = qb.State(circ.dims, prec=qb.QD_C64)
    st.run(circ, fuse=fuse)
    mid = st.norm()
    st.run(inv, fuse=fuse)
    nrm = st.norm()
    amp0 = st.buf[:2].double().cpu().numpy()
    st.close()
    del st
    torch.cuda.empty_cache()
    p0 = float(amp0[0] ** 2 + amp0[1] ** 2)
    assert abs(mid - 1.0) < 1e-4
    assert abs(nrm - 1.0) < 1e-4
    assert p0 > 1.0 - 1e-4, f"|psi_0|^2 = {p0}"
    assert 1.0 - p0 / nrm < 1e-4
