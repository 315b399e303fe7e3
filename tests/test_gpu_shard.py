"""GPU side of the partitioned state: the wire move of the exchange step
(qd_state_wire_to_top / qd_state_wire_from_top) against numpy's reshape and
transpose of the same amplitudes, every wire of ragged mixed-radix layouts
in both precisions, bit for bit (the move copies values)."""
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
@pytest.mark.parametrize("dims", [(2, 3, 4, 5, 2, 3), (5,), (3, 2, 2, 2, 2, 2, 2, 2, 3, 3, 2, 5, 7)])
def test_wire_move_against_numpy(qb, prec, dims):
    import torch

    from paper_2410_17876_gb300 import inputs as gen

    p = qb.QD_C64 if prec == "c64" else qb.QD_C128
    rng = np.random.Generator(np.random.PCG64(len(dims)))
    st = qb.State(dims, prec=p)
    st.set_amplitudes(gen.random_state(st.D, rng))
    psi = st.raw().copy()
    out = torch.empty_like(st.buf)
    for w in range(len(dims)):
        lo = int(np.prod(dims[:w], dtype=np.int64))
        d = dims[w]
        hi = st.D // (lo * d)
        qb.qd_state_wire_to_top(st.handle, w, out.data_ptr())
        st.synchronize()
        got = out.cpu().numpy().view(psi.dtype)
        want = np.ascontiguousarray(psi.reshape(hi, d, lo).transpose(1, 0, 2)).reshape(-1)
        assert np.array_equal(got, want), (dims, w)
        # and back: the state set from the moved order is the original state
        st.reset()
        qb.qd_state_wire_from_top(st.handle, w, out.data_ptr())
        assert np.array_equal(st.raw(), psi), (dims, w)
    with pytest.raises(qb.QuditError):
        qb.qd_state_wire_to_top(st.handle, len(dims), out.data_ptr())
    with pytest.raises(qb.QuditError):
        qb.qd_state_wire_to_top(st.handle, 0, st.buf.data_ptr())  # overlaps the state
    st.close()
