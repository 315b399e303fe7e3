"""Checkpoint and resume of a state (qd_state_save / qd_state_load): the
same bits after a round trip through a file, across more than one staging
chunk, with queued deferred gates applied first; a file of other dims is
rejected before anything is read, a short file is rejected."""
import numpy as np
import pytest

import __graft_entry__

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qb():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    __graft_entry__.build()
    from paper_2410_17876_gb300 import binding

    return binding


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_round_trip_is_bit_exact(qb, tmp_path, prec):
    from paper_2410_17876_gb300 import inputs as gen

    p = qb.QD_C64 if prec == "c64" else qb.QD_C128
    rng = np.random.Generator(np.random.PCG64(9))
    dims = (2,) * 21 + (3, 2, 2, 2)  # 50.3M amplitudes: 403 MB / 805 MB, more than one 256 MiB chunk
    circ = gen.random_mixed_circuit(dims, 40, rng)
    st = qb.State(dims, prec=p)
    st.run(circ, fuse="tile")
    st.set_fusion(4)                 # a deferred gate still queued when the state is saved
    st.apply(circ.gates[0])
    f = tmp_path / "state.qd"
    qb.qd_state_save(st.handle, str(f))
    want = st.raw().copy()           # the queued gate was applied by the save
    st.reset()
    qb.qd_state_load(st.handle, str(f))
    assert np.array_equal(st.raw(), want)
    other = qb.State(dims[:-1], prec=p)
    before = other.raw().copy()
    with pytest.raises(qb.QuditError):
        qb.qd_state_load(other.handle, str(f))
    assert np.array_equal(other.raw(), before)
    other.close()
    short = tmp_path / "short.qd"
    short.write_bytes(f.read_bytes()[: 1 << 20])
    st.reset()
    with pytest.raises(qb.QuditError):
        qb.qd_state_load(st.handle, str(short))
    st.close()
